"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never calls
it and shares no code with it.

Every function is a thin ctypes wrapper around ``mrioracle.c``, a plain
double-precision direct-summation implementation of the paper's operators:

* :func:`forward`   -- Eq. 1-2, multi-coil non-uniform DFT by direct summation
* :func:`adjoint`   -- its adjoint, coil combination included
* :func:`tv_forward` / :func:`tv_adjoint` -- the finite-difference sparsifying
  transform Theta of Eq. 3 and its transpose
* :func:`shrink`    -- soft threshold, Eq. 8-9
* :func:`normal`    -- Eq. 11, ``F^H F + (beta/2) Theta^H Theta``
* :func:`cg`        -- Alg. 2
* :func:`objective` -- Eq. 3
* :func:`admm`      -- Alg. 4 with Eq. 6-12

Arrays are numpy complex128 in the library layouts: image ``[nx][ny]``, coil
maps ``[nc][nx][ny]``, k-space ``[nc][nk]``, trajectory ``[nk][2]`` (float64
of the float32 values the GPU sees), Theta output ``[2][nx][ny]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mrioracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``mrioracle.c`` into ``liboracle.so`` (gcc, OpenMP, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.orc_forward.argtypes = [I, I, I, I, P, P, P, P]
        lib.orc_adjoint.argtypes = [I, I, I, I, P, P, P, P]
        lib.orc_adjoint_at.argtypes = [I, I, I, I, P, P, P, I, P, P]
        lib.orc_tv_forward.argtypes = [I, I, P, P]
        lib.orc_tv_adjoint.argtypes = [I, I, P, P]
        lib.orc_shrink.argtypes = [I, D, P, P]
        lib.orc_normal.argtypes = [I, I, I, I, P, P, D, P, P]
        lib.orc_cg.argtypes = [I, I, I, I, P, P, D, P, P, I, D, P]
        lib.orc_cg.restype = I
        lib.orc_objective.argtypes = [I, I, I, I, P, P, P, D, P]
        lib.orc_objective.restype = D
        lib.orc_admm.argtypes = [I, I, I, I, P, P, P, D, D, I, I, D, D, P, P, P, P, P]
        lib.orc_admm.restype = I
        lib.orc_set_threads.argtypes = [I]
        lib.orc_get_threads.restype = I
        _lib = lib
    return _lib


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def forward(traj, image, maps):
    """Eq. 1: ``d[c][kappa] = sum_n S_c[n] x[n] exp(-i 2 pi k_kappa . r_n)``."""
    lib = _load()
    traj = _c(traj, np.float64)
    image = _c(image)
    maps = _c(maps)
    nc, nx, ny = maps.shape
    nk = traj.shape[0]
    out = np.empty((nc, nk), np.complex128)
    lib.orc_forward(nx, ny, nk, nc, _p(traj), _p(image), _p(maps), _p(out))
    return out


def adjoint(traj, kspace, maps):
    """Adjoint of Eq. 1: ``x[n] = sum_c conj(S_c[n]) sum_kappa d_c[kappa] exp(+i 2 pi k.r_n)``."""
    lib = _load()
    traj = _c(traj, np.float64)
    kspace = _c(kspace)
    maps = _c(maps)
    nc, nx, ny = maps.shape
    nk = traj.shape[0]
    out = np.empty((nx, ny), np.complex128)
    lib.orc_adjoint(nx, ny, nk, nc, _p(traj), _p(kspace), _p(maps), _p(out))
    return out


def adjoint_at(traj, kspace, maps, pixels):
    """The adjoint of Eq. 1 at the flat pixel indices ``pixels`` (``i*ny + j``) only."""
    lib = _load()
    traj = _c(traj, np.float64)
    kspace = _c(kspace)
    maps = _c(maps)
    pix = np.ascontiguousarray(pixels, dtype=np.int32)
    nc, nx, ny = maps.shape
    out = np.empty(pix.size, np.complex128)
    lib.orc_adjoint_at(nx, ny, traj.shape[0], nc, _p(traj), _p(kspace), _p(maps), int(pix.size), _p(pix),
                       _p(out))
    return out


def tv_forward(image):
    """Theta: forward differences along both axes, zero past the last pixel; ``[2][nx][ny]``."""
    lib = _load()
    image = _c(image)
    nx, ny = image.shape
    out = np.empty((2, nx, ny), np.complex128)
    lib.orc_tv_forward(nx, ny, _p(image), _p(out))
    return out


def tv_adjoint(grad):
    """Theta^H, the transpose of :func:`tv_forward`."""
    lib = _load()
    grad = _c(grad)
    _, nx, ny = grad.shape
    out = np.empty((nx, ny), np.complex128)
    lib.orc_tv_adjoint(nx, ny, _p(grad), _p(out))
    return out


def shrink(a, t: float):
    """Eq. 8-9 soft threshold for complex values: ``a (1 - t/|a|)`` if ``|a| > t`` else 0."""
    lib = _load()
    a = _c(a)
    out = np.empty_like(a)
    lib.orc_shrink(a.size, float(t), _p(a), _p(out))
    return out


def normal(traj, maps, beta: float, p):
    """Eq. 11: ``F^H F p + (beta/2) Theta^H Theta p``."""
    lib = _load()
    traj = _c(traj, np.float64)
    maps = _c(maps)
    p = _c(p)
    nc, nx, ny = maps.shape
    out = np.empty((nx, ny), np.complex128)
    lib.orc_normal(nx, ny, traj.shape[0], nc, _p(traj), _p(maps), float(beta), _p(p), _p(out))
    return out


def cg(traj, maps, beta: float, b, x0, max_iter: int, atol: float = 0.0):
    """Alg. 2.  Returns ``(x, steps, tau_history)``."""
    lib = _load()
    traj = _c(traj, np.float64)
    maps = _c(maps)
    b = _c(b)
    x = _c(x0).copy()
    nc, nx, ny = maps.shape
    hist = np.zeros(max_iter + 1, np.float64)
    steps = lib.orc_cg(nx, ny, traj.shape[0], nc, _p(traj), _p(maps), float(beta), _p(b), _p(x),
                       int(max_iter), float(atol), _p(hist))
    return x, int(steps), hist[: steps + 1]


def objective(traj, maps, kspace, lam: float, image) -> float:
    """Eq. 3: ``||F x - d||^2 + lambda * sum |Theta x|``."""
    lib = _load()
    traj = _c(traj, np.float64)
    maps = _c(maps)
    kspace = _c(kspace)
    image = _c(image)
    nc, nx, ny = maps.shape
    return float(lib.orc_objective(nx, ny, traj.shape[0], nc, _p(traj), _p(maps), _p(kspace),
                                   float(lam), _p(image)))


def admm(traj, maps, kspace, lam: float, beta: float, admm_iters: int, cg_iters: int,
         rtol: float = 0.0, atol: float = 0.0, want_state: bool = False):
    """Alg. 4.  Returns a dict with ``x``, ``steps``, ``objective`` and ``alpha``
    histories (and ``mu``, ``eta`` when ``want_state``)."""
    lib = _load()
    traj = _c(traj, np.float64)
    maps = _c(maps)
    kspace = _c(kspace)
    nc, nx, ny = maps.shape
    x = np.zeros((nx, ny), np.complex128)
    obj = np.zeros(max(admm_iters, 1), np.float64)
    alpha = np.zeros(max(admm_iters, 1), np.float64)
    mu = np.zeros((2, nx, ny), np.complex128)
    eta = np.zeros((2, nx, ny), np.complex128)
    steps = lib.orc_admm(nx, ny, traj.shape[0], nc, _p(traj), _p(maps), _p(kspace), float(lam),
                         float(beta), int(admm_iters), int(cg_iters), float(rtol), float(atol),
                         _p(x), _p(obj), _p(alpha), _p(mu), _p(eta))
    out = {"x": x, "steps": int(steps), "objective": obj[:steps], "alpha": alpha[:steps]}
    if want_state:
        out["mu"] = mu
        out["eta"] = eta
    return out


def measurements(problem) -> np.ndarray:
    """Noisy k-space for a :class:`synth.Problem`: the oracle's forward model of
    the phantom plus the problem's seeded noise, rounded to complex64."""
    import synth
    d_clean = forward(problem.traj, problem.image_true, problem.maps)
    return synth.add_noise(d_clean, problem.noise, problem.noise_level)
