"""Python binding of libmrirecon (GB300 / sm_103a MRI reconstruction).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libmrirecon.so``.  PyTorch supplies device memory and the current
stream.  The functions mirror the C entry points of ``include/mrirecon.h``:

* :class:`Plan`            -- ``mri_plan_create`` / ``mri_plan_set_trajectory`` /
  ``mri_plan_destroy`` (DFT factor generation, Alg. 1)
* :func:`nudft_forward`    -- Eq. 1-2
* :func:`nudft_adjoint`    -- adjoint of Eq. 1 with coil combination
* :func:`normal_op`        -- Eq. 11
* :func:`tv_forward`, :func:`tv_adjoint` -- the finite-difference transform Theta
* :func:`soft_threshold`   -- Eq. 9
* :func:`admm_reconstruct` -- Alg. 4
* :class:`Batch`           -- many reconstructions in one launch
* :class:`Server`          -- requests from host memory under a device-memory budget

Tensors are CUDA, contiguous, complex64 (images ``[nx, ny]``, coil maps
``[nc, nx, ny]``, k-space ``[nc, nk]``) or float32 (trajectory ``[nk, 2]``).
If the shared library is missing the import fails loudly: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmrirecon.so")

MRI_OK = 0
MRI_ERR_INVALID = -1
MRI_ERR_NOMEM = -2
MRI_ERR_CUDA = -3
MRI_ERR_TIMEOUT = -4
MRI_ERR_UNSUPPORTED = -5

MRI_FP32 = 0
MRI_TF32 = 1
MRI_BF16X3 = 2
PRECISIONS = {"fp32": MRI_FP32, "tf32": MRI_TF32, "bf16x3": MRI_BF16X3}


class MriError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"mrirecon error {code}: {msg}")
        self.code = code


class AdmmParams(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_float), ("beta", ctypes.c_float), ("admm_iters", ctypes.c_int),
                ("cg_iters", ctypes.c_int), ("rtol", ctypes.c_double), ("atol", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("kspace", ctypes.c_void_p), ("coil_maps", ctypes.c_void_p),
                ("image_out", ctypes.c_void_p), ("params", AdmmParams)]


class ServerRequest(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nk", ctypes.c_int), ("nc", ctypes.c_int),
                ("traj", ctypes.c_void_p), ("kspace", ctypes.c_void_p), ("coil_maps", ctypes.c_void_p),
                ("params", AdmmParams)]


_lib = None


def load(path: str = LIB_PATH):
    """Load ``libmrirecon.so``; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmrirecon.so not built ({path}); run paper_2006_14080_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, F, D, Z = ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double, ctypes.c_size_t
    sigs = {
        "mri_last_error": ([], ctypes.c_char_p),
        "mri_version": ([], I),
        "mri_plan_create": ([ctypes.POINTER(P), I, I, I, I, P, I, P], I),
        "mri_plan_set_trajectory": ([P, P, P], I),
        "mri_plan_destroy": ([P], I),
        "mri_plan_sync_status": ([P, P], I),
        "mri_plan_device_bytes": ([P], Z),
        "mri_plan_estimate_bytes": ([I, I, I, I, I], Z),
        "mri_nudft_forward": ([P, P, P, P, P], I),
        "mri_nudft_adjoint": ([P, P, P, P, P], I),
        "mri_normal_op": ([P, P, P, F, P, P], I),
        "mri_tv_forward": ([I, I, P, P, P], I),
        "mri_tv_adjoint": ([I, I, P, P, P], I),
        "mri_soft_threshold": ([I, F, P, P, P], I),
        "mri_admm_reconstruct": ([P, P, P, ctypes.POINTER(AdmmParams), P, P, P, P], I),
        "mri_admm_resume": ([P, P, P, ctypes.POINTER(AdmmParams), P, P, P, P, P, P, P], I),
        "mri_nudft_adjoint_noalloc": ([I, I, I, I, P, P, P, P, P], I),
        "mri_plan_set_timing": ([P, I], I),
        "mri_plan_read_timing": ([P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                  ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(D),
                                  ctypes.POINTER(ctypes.c_longlong)], I),
        "mri_plan_launch_count": ([P], ctypes.c_longlong),
        "mri_plan_selftest_wait": ([P, D, P], I),
        "mri_plan_get_config": ([P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "mri_plan_set_tiles": ([P, I, I, I], I),
        "mri_plan_autotune": ([P, I, P], I),
        "mri_plan_set_graphs": ([P, I], I),
        "mri_batch_create": ([ctypes.POINTER(P)], I),
        "mri_batch_destroy": ([P], I),
        "mri_batch_reconstruct": ([P, I, ctypes.POINTER(Request), P], I),
        "mri_batch_launch_count": ([P], ctypes.c_longlong),
        "mri_server_create": ([ctypes.POINTER(P), Z, I, I], I),
        "mri_server_submit": ([P, ctypes.POINTER(ServerRequest), ctypes.POINTER(ctypes.c_uint64)], I),
        "mri_server_poll": ([P, ctypes.c_uint64, ctypes.POINTER(I)], I),
        "mri_server_wait": ([P, ctypes.c_uint64, P, ctypes.POINTER(D), D], I),
        "mri_server_stats": ([P, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(Z), ctypes.POINTER(Z)], I),
        "mri_server_cache_stats": ([P] + [ctypes.POINTER(ctypes.c_uint64)] * 4, I),
        "mri_server_destroy": ([P], I),
        "mri_tuning_save": ([ctypes.c_char_p], I),
        "mri_tuning_load": ([ctypes.c_char_p], I),
        "mri_tuning_clear": ([], I),
        "mri_tuning_count": ([], I),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int):
    if rc != MRI_OK:
        raise MriError(rc, load().mri_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, shape, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Plan:
    """DFT factors for one trajectory plus all workspace (``mri_plan``)."""

    def __init__(self, nx: int, ny: int, nc: int, traj: torch.Tensor, precision: str = "bf16x3", stream=None):
        lib = load()
        nk = int(traj.shape[0])
        _need(traj, torch.float32, (nk, 2), "traj")
        self.nx, self.ny, self.nc, self.nk = int(nx), int(ny), int(nc), nk
        self.precision = precision
        h = ctypes.c_void_p()
        _check(lib.mri_plan_create(ctypes.byref(h), self.nx, self.ny, nk, self.nc, _ptr(traj),
                                   PRECISIONS[precision], _stream(stream)))
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan is closed")
        return self._h

    def set_trajectory(self, traj: torch.Tensor, stream=None):
        _need(traj, torch.float32, (self.nk, 2), "traj")
        _check(load().mri_plan_set_trajectory(self.handle, _ptr(traj), _stream(stream)))

    def sync_status(self, stream=None):
        _check(load().mri_plan_sync_status(self.handle, _stream(stream)))

    def device_bytes(self) -> int:
        return int(load().mri_plan_device_bytes(self.handle))

    def set_timing(self, enable: bool = True):
        _check(load().mri_plan_set_timing(self.handle, int(bool(enable))))

    def read_timing(self):
        """``{"fwd_ms", "fwd_launches", "adj_ms", "adj_launches", "red_ms", "red_launches"}``
        since the last read."""
        fm, am, rm = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        fn, an, rn = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
        _check(load().mri_plan_read_timing(self.handle, ctypes.byref(fm), ctypes.byref(fn), ctypes.byref(am),
                                           ctypes.byref(an), ctypes.byref(rm), ctypes.byref(rn)))
        return {"fwd_ms": fm.value, "fwd_launches": fn.value, "adj_ms": am.value, "adj_launches": an.value,
                "red_ms": rm.value, "red_launches": rn.value}

    def launch_count(self) -> int:
        return int(load().mri_plan_launch_count(self.handle))

    def selftest_wait(self, limit_ms: float, stream=None):
        """Enqueue a bounded wait that runs out after ``limit_ms`` (failure-detection self-test)."""
        _check(load().mri_plan_selftest_wait(self.handle, float(limit_ms), _stream(stream)))

    def config(self) -> dict:
        v = [ctypes.c_int() for _ in range(4)]
        _check(load().mri_plan_get_config(self.handle, *[ctypes.byref(q) for q in v]))
        return {"fwd_coils_per_tile": v[0].value, "fwd_stages": v[1].value, "adj_stages": v[2].value,
                "adj_ksplit": v[3].value}

    def set_graphs(self, enable: bool = True):
        """Capture/replay whole reconstructions as CUDA graphs (default on)."""
        _check(load().mri_plan_set_graphs(self.handle, int(bool(enable))))

    def set_tiles(self, fwd_coils_per_tile: int = 0, fwd_stages: int = 0, adj_stages: int = 0):
        """Tile configuration of the tensor-core products (0 keeps the current value)."""
        _check(load().mri_plan_set_tiles(self.handle, int(fwd_coils_per_tile), int(fwd_stages), int(adj_stages)))

    def autotune(self, repeats: int = 3, stream=None) -> dict:
        """Time the valid tile configurations of both products on this shape and keep the fastest."""
        _check(load().mri_plan_autotune(self.handle, int(repeats), _stream(stream)))
        return self.config()

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().mri_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def nudft_forward(plan: Plan, image, coil_maps, out=None, stream=None):
    _need(image, torch.complex64, (plan.nx, plan.ny), "image")
    _need(coil_maps, torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
    if out is None:
        out = torch.empty((plan.nc, plan.nk), dtype=torch.complex64, device=image.device)
    _need(out, torch.complex64, (plan.nc, plan.nk), "kspace")
    _check(load().mri_nudft_forward(plan.handle, _ptr(image), _ptr(coil_maps), _ptr(out), _stream(stream)))
    return out


def nudft_adjoint(plan: Plan, kspace, coil_maps, out=None, stream=None):
    _need(kspace, torch.complex64, (plan.nc, plan.nk), "kspace")
    _need(coil_maps, torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
    if out is None:
        out = torch.empty((plan.nx, plan.ny), dtype=torch.complex64, device=kspace.device)
    _need(out, torch.complex64, (plan.nx, plan.ny), "image")
    _check(load().mri_nudft_adjoint(plan.handle, _ptr(kspace), _ptr(coil_maps), _ptr(out), _stream(stream)))
    return out


def nudft_adjoint_noalloc(traj, kspace, coil_maps, out, stream=None):
    """Adjoint DFT without a plan and without any device allocation by the
    library (``mri_nudft_adjoint_noalloc``): for callers that must not touch
    the CUDA allocator.  ``out`` is required (the caller owns all memory)."""
    nc, nx, ny = coil_maps.shape
    nk = traj.shape[0]
    _need(traj, torch.float32, (nk, 2), "traj")
    _need(kspace, torch.complex64, (nc, nk), "kspace")
    _need(coil_maps, torch.complex64, (nc, nx, ny), "coil_maps")
    _need(out, torch.complex64, (nx, ny), "image")
    _check(load().mri_nudft_adjoint_noalloc(nx, ny, nk, nc, _ptr(traj), _ptr(kspace), _ptr(coil_maps), _ptr(out),
                                            _stream(stream)))
    return out


def normal_op(plan: Plan, image, coil_maps, beta: float = 0.0, out=None, stream=None):
    _need(image, torch.complex64, (plan.nx, plan.ny), "image")
    _need(coil_maps, torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
    if out is None:
        out = torch.empty_like(image)
    _need(out, torch.complex64, (plan.nx, plan.ny), "out")
    _check(load().mri_normal_op(plan.handle, _ptr(image), _ptr(coil_maps), float(beta), _ptr(out),
                                _stream(stream)))
    return out


def tv_forward(image, out=None, stream=None):
    nx, ny = image.shape
    _need(image, torch.complex64, (nx, ny), "image")
    if out is None:
        out = torch.empty((2, nx, ny), dtype=torch.complex64, device=image.device)
    _need(out, torch.complex64, (2, nx, ny), "grad")
    _check(load().mri_tv_forward(nx, ny, _ptr(image), _ptr(out), _stream(stream)))
    return out


def tv_adjoint(grad, out=None, stream=None):
    _, nx, ny = grad.shape
    _need(grad, torch.complex64, (2, nx, ny), "grad")
    if out is None:
        out = torch.empty((nx, ny), dtype=torch.complex64, device=grad.device)
    _need(out, torch.complex64, (nx, ny), "image")
    _check(load().mri_tv_adjoint(nx, ny, _ptr(grad), _ptr(out), _stream(stream)))
    return out


def soft_threshold(x, t: float, out=None, stream=None):
    _need(x, torch.complex64, tuple(x.shape), "x")
    if out is None:
        out = torch.empty_like(x)
    _need(out, torch.complex64, tuple(x.shape), "out")
    _check(load().mri_soft_threshold(x.numel(), float(t), _ptr(x), _ptr(out), _stream(stream)))
    return out


def admm_reconstruct(plan: Plan, kspace, coil_maps, lam: float, beta: float, admm_iters: int, cg_iters: int,
                     rtol: float = 0.0, atol: float = 0.0, out=None, objective_hist=None, alpha_hist=None,
                     stream=None):
    """Alg. 4.  ``objective_hist`` / ``alpha_hist``: optional CUDA float64
    tensors of ``admm_iters`` entries that receive the Eq. 3 objective and the
    relative change after each outer step."""
    _need(kspace, torch.complex64, (plan.nc, plan.nk), "kspace")
    _need(coil_maps, torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
    if out is None:
        out = torch.empty((plan.nx, plan.ny), dtype=torch.complex64, device=kspace.device)
    _need(out, torch.complex64, (plan.nx, plan.ny), "image_out")
    for h, name in ((objective_hist, "objective_hist"), (alpha_hist, "alpha_hist")):
        if h is not None:
            _need(h, torch.float64, (admm_iters,), name)
    prm = AdmmParams(float(lam), float(beta), int(admm_iters), int(cg_iters), float(rtol), float(atol))
    _check(load().mri_admm_reconstruct(plan.handle, _ptr(kspace), _ptr(coil_maps), ctypes.byref(prm), _ptr(out),
                                       _ptr(objective_hist), _ptr(alpha_hist), _stream(stream)))
    return out


def admm_resume(plan: Plan, kspace, coil_maps, lam: float, beta: float, admm_iters: int, cg_iters: int,
                x0=None, eta0=None, rtol: float = 0.0, atol: float = 0.0, out=None, eta_out=None,
                objective_hist=None, alpha_hist=None, stream=None):
    """Alg. 4 from a saved state (``mri_admm_resume``): ``x0`` ``[nx, ny]`` and
    ``eta0`` ``[2, nx, ny]`` (None: zero).  Returns ``(image, eta)``; ``eta`` is
    a new tensor unless ``eta_out`` is given."""
    _need(kspace, torch.complex64, (plan.nc, plan.nk), "kspace")
    _need(coil_maps, torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
    if x0 is not None:
        _need(x0, torch.complex64, (plan.nx, plan.ny), "x0")
    if eta0 is not None:
        _need(eta0, torch.complex64, (2, plan.nx, plan.ny), "eta0")
    if out is None:
        out = torch.empty((plan.nx, plan.ny), dtype=torch.complex64, device=kspace.device)
    if eta_out is None:
        eta_out = torch.empty((2, plan.nx, plan.ny), dtype=torch.complex64, device=kspace.device)
    _need(out, torch.complex64, (plan.nx, plan.ny), "image_out")
    _need(eta_out, torch.complex64, (2, plan.nx, plan.ny), "eta_out")
    for h, name in ((objective_hist, "objective_hist"), (alpha_hist, "alpha_hist")):
        if h is not None:
            _need(h, torch.float64, (admm_iters,), name)
    prm = AdmmParams(float(lam), float(beta), int(admm_iters), int(cg_iters), float(rtol), float(atol))
    _check(load().mri_admm_resume(plan.handle, _ptr(kspace), _ptr(coil_maps), ctypes.byref(prm), _ptr(x0),
                                  _ptr(eta0), _ptr(out), _ptr(eta_out), _ptr(objective_hist), _ptr(alpha_hist),
                                  _stream(stream)))
    return out, eta_out


class Batch:
    """Many independent reconstructions in one launch (``mri_batch_*``).

    ``reconstruct(items)`` takes a list of dicts with keys ``plan``, ``kspace``,
    ``coil_maps``, ``out`` (CUDA tensors as for :func:`admm_reconstruct`) and
    ``lam``, ``beta``, ``admm_iters``, ``cg_iters`` (optional ``rtol``,
    ``atol``).  Each item needs its own plan.  The combined launch is cached
    while the item list repeats.
    """

    def __init__(self):
        h = ctypes.c_void_p()
        _check(load().mri_batch_create(ctypes.byref(h)))
        self._h = h
        self._keep = None

    def reconstruct(self, items, stream=None):
        reqs = (Request * len(items))()
        for q, it in enumerate(items):
            plan = it["plan"]
            _need(it["kspace"], torch.complex64, (plan.nc, plan.nk), "kspace")
            _need(it["coil_maps"], torch.complex64, (plan.nc, plan.nx, plan.ny), "coil_maps")
            _need(it["out"], torch.complex64, (plan.nx, plan.ny), "out")
            reqs[q].plan = plan.handle.value
            reqs[q].kspace = it["kspace"].data_ptr()
            reqs[q].coil_maps = it["coil_maps"].data_ptr()
            reqs[q].image_out = it["out"].data_ptr()
            reqs[q].params = AdmmParams(float(it["lam"]), float(it["beta"]), int(it["admm_iters"]),
                                        int(it["cg_iters"]), float(it.get("rtol", 0.0)), float(it.get("atol", 0.0)))
        self._keep = items  # the cached launch refers to these tensors
        _check(load().mri_batch_reconstruct(self._h, len(items), reqs, _stream(stream)))

    def launch_count(self) -> int:
        return int(load().mri_batch_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().mri_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def estimate_plan_bytes(nx: int, ny: int, nk: int, nc: int, precision: str = "bf16x3") -> int:
    """Device bytes a plan of this shape would hold (``mri_plan_estimate_bytes``)."""
    return int(load().mri_plan_estimate_bytes(nx, ny, nk, nc, PRECISIONS[precision]))


class Server:
    """Serving loop (``mri_server_*``): requests from HOST arrays, admitted under
    a device-memory budget and run concurrently on ``max_inflight`` streams.

    ``submit`` takes numpy arrays (or CPU tensors): ``traj`` float32
    ``[nk, 2]``, ``kspace`` complex64 ``[nc, nk]``, ``coil_maps`` complex64
    ``[nc, nx, ny]``; it copies them and returns a ticket.  ``wait(ticket)``
    returns ``(image, latency_ms)`` with ``image`` a complex64 numpy array
    ``[nx, ny]``, or raises :class:`MriError` with the request's status.
    """

    def __init__(self, budget_bytes: int, max_inflight: int = 4, precision: str = "bf16x3"):
        h = ctypes.c_void_p()
        _check(load().mri_server_create(ctypes.byref(h), int(budget_bytes), int(max_inflight),
                                        PRECISIONS[precision]))
        self._h = h
        self._shapes = {}

    def submit(self, traj, kspace, coil_maps, lam: float, beta: float, admm_iters: int, cg_iters: int,
               rtol: float = 0.0, atol: float = 0.0) -> int:
        import numpy as np
        traj = np.ascontiguousarray(np.asarray(traj), dtype=np.float32)
        kspace = np.ascontiguousarray(np.asarray(kspace), dtype=np.complex64)
        coil_maps = np.ascontiguousarray(np.asarray(coil_maps), dtype=np.complex64)
        nc, nx, ny = coil_maps.shape
        nk = traj.shape[0]
        if traj.shape != (nk, 2) or kspace.shape != (nc, nk):
            raise ValueError(f"inconsistent shapes: traj {traj.shape}, kspace {kspace.shape}, maps {coil_maps.shape}")
        req = ServerRequest(nx, ny, nk, nc, traj.ctypes.data, kspace.ctypes.data, coil_maps.ctypes.data,
                            AdmmParams(float(lam), float(beta), int(admm_iters), int(cg_iters), float(rtol),
                                       float(atol)))
        t = ctypes.c_uint64()
        _check(load().mri_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        self._shapes[t.value] = (nx, ny)
        return t.value

    def poll(self, ticket: int) -> bool:
        done = ctypes.c_int()
        _check(load().mri_server_poll(self._h, ticket, ctypes.byref(done)))
        return bool(done.value)

    def wait(self, ticket: int, timeout_s: float = 0.0):
        import numpy as np
        nx, ny = self._shapes[ticket]
        img = np.empty((nx, ny), dtype=np.complex64)
        lat = ctypes.c_double()
        rc = load().mri_server_wait(self._h, ticket, img.ctypes.data, ctypes.byref(lat), float(timeout_s))
        if rc != MRI_ERR_TIMEOUT or timeout_s <= 0:
            self._shapes.pop(ticket, None)
        _check(rc)
        return img, lat.value

    def stats(self) -> dict:
        p50, p99 = ctypes.c_double(), ctypes.c_double()
        done, failed = ctypes.c_uint64(), ctypes.c_uint64()
        res, peak = ctypes.c_size_t(), ctypes.c_size_t()
        _check(load().mri_server_stats(self._h, ctypes.byref(p50), ctypes.byref(p99), ctypes.byref(done),
                                       ctypes.byref(failed), ctypes.byref(res), ctypes.byref(peak)))
        c = [ctypes.c_uint64() for _ in range(4)]
        _check(load().mri_server_cache_stats(self._h, *[ctypes.byref(q) for q in c]))
        return {"p50_ms": p50.value, "p99_ms": p99.value, "completed": done.value, "failed": failed.value,
                "resident_bytes": res.value, "peak_resident_bytes": peak.value, "plan_hits": c[0].value,
                "plan_retargets": c[1].value, "maps_reused": c[2].value, "graph_replays": c[3].value}

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().mri_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tuning_save(path: str):
    """Write the autotuning table (``mri_tuning_save``)."""
    _check(load().mri_tuning_save(os.fsencode(path)))


def tuning_load(path: str):
    """Merge a saved autotuning table (``mri_tuning_load``)."""
    _check(load().mri_tuning_load(os.fsencode(path)))


def tuning_clear():
    _check(load().mri_tuning_clear())


def tuning_count() -> int:
    return int(load().mri_tuning_count())
