"""Seeded synthetic inputs for the multi-coil radial MRI reconstruction.

This module is shared by the FP64 oracle tests and the GPU path.  It draws
random numbers and lays out arrays; it contains none of the reconstruction
arithmetic (no Fourier encoding, no finite differences, no thresholding, no
solver).  The k-space measurement ``d`` is therefore *not* produced here: the
caller applies its own forward operator to ``image_true`` and then calls
:func:`add_noise` with the unit noise drawn here.

Recipe (the paper's scanner phantom data are not available; these inputs stand
in for them with the same structure: multi-coil, radial spokes, 2x oversampled
readouts, undersampled angles):

* trajectory: spoke ``s`` of ``S``, readout sample ``r`` of ``R``;
  ``k_r = (r - R/2)/R`` cycles/pixel, angle ``pi*s/S`` (uniform) or
  ``s*pi*(sqrt(5)-1)/2`` (golden angle); sample index ``kappa = s*R + r``.
* coil maps: Gaussian blobs centred on an ellipse of radius ``0.5*(Nx, Ny)``
  at angle ``2*pi*c/C``, width ``0.4*N``, seeded constant phase, normalised so
  that ``sum_c |S_c|^2 = 1`` at every pixel.
* phantom: 10 ellipses, the first a body ellipse of intensity 1, the others
  with seeded centre (uniform in a disk of radius ``0.35*N``), semi-axes
  ``U[0.05, 0.3]*N``, angle ``U[0, pi)`` and additive intensity
  ``U[-0.4, 1]``; rasterised by pixel-centre inclusion (or by an
  ``ss x ss`` supersampled coverage fraction).
* noise: circular complex Gaussian with unit variance (1/2 per component);
  scaled by ``p * RMS(|d_clean|)`` in :func:`add_noise`.

Pixel coordinates are integers centred on the grid: ``x_i = i - Nx//2``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GOLDEN_ANGLE = math.pi * (math.sqrt(5.0) - 1.0) / 2.0  # ~111.246 degrees


def pixel_coords(n: int) -> np.ndarray:
    """Integer pixel-centre coordinates ``i - n//2`` for ``i = 0..n-1``."""
    return np.arange(n, dtype=np.float64) - (n // 2)


def radial_trajectory(spokes: int, readout: int, golden: bool = True, rotation: float = 0.0) -> np.ndarray:
    """Radial k-space trajectory, float32 ``[spokes*readout][2]`` in cycles/pixel;
    every spoke angle is offset by ``rotation`` radians."""
    r = (np.arange(readout, dtype=np.float64) - readout / 2.0) / readout
    if golden:
        theta = rotation + np.arange(spokes, dtype=np.float64) * GOLDEN_ANGLE
    else:
        theta = rotation + np.arange(spokes, dtype=np.float64) * (math.pi / spokes)
    kx = np.outer(np.cos(theta), r).reshape(-1)
    ky = np.outer(np.sin(theta), r).reshape(-1)
    return np.stack([kx, ky], axis=1).astype(np.float32)


def cartesian_trajectory(nx: int, ny: int, dtype=np.float32) -> np.ndarray:
    """All ``nx*ny`` Cartesian grid frequencies ``((m - nx//2)/nx, (l - ny//2)/ny)``,
    ordered with the second index fastest; ``[nx*ny][2]`` (float32 unless
    ``dtype`` says otherwise: ``m/nx`` is exact in float32 only for powers of two)."""
    kx = (np.arange(nx) - nx // 2) / nx
    ky = (np.arange(ny) - ny // 2) / ny
    KX, KY = np.meshgrid(kx, ky, indexing="ij")
    return np.stack([KX.reshape(-1), KY.reshape(-1)], axis=1).astype(dtype)


@dataclasses.dataclass
class Ellipse:
    cx: float
    cy: float
    a: float        # semi-axis along the rotated x direction
    b: float        # semi-axis along the rotated y direction
    angle: float    # rotation in radians
    value: float    # additive intensity


def random_ellipses(rng: np.random.Generator, nx: int, ny: int, count: int = 10) -> List[Ellipse]:
    n = float(min(nx, ny))
    out = [Ellipse(0.0, 0.0, 0.40 * nx, 0.34 * ny, float(rng.uniform(0.0, math.pi)), 1.0)]
    for _ in range(count - 1):
        rad = 0.35 * n * math.sqrt(rng.uniform())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        a = rng.uniform(0.05, 0.3) * n
        b = rng.uniform(0.05, 0.3) * n
        ang = rng.uniform(0.0, math.pi)
        val = rng.uniform(-0.4, 1.0)
        out.append(Ellipse(rad * math.cos(phi), rad * math.sin(phi), a, b, ang, val))
    return out


def rasterize(ellipses: Sequence[Ellipse], nx: int, ny: int, ss: int = 1) -> np.ndarray:
    """Sum of ellipse indicators sampled on the pixel grid; with ``ss > 1`` each
    pixel holds the covered fraction of an ``ss x ss`` sub-grid.  complex64."""
    off = (np.arange(ss) + 0.5) / ss - 0.5
    X = (pixel_coords(nx)[:, None] + off[None, :]).reshape(-1)
    Y = (pixel_coords(ny)[:, None] + off[None, :]).reshape(-1)
    XX, YY = np.meshgrid(X, Y, indexing="ij")
    img = np.zeros_like(XX)
    for e in ellipses:
        c, s = math.cos(e.angle), math.sin(e.angle)
        u = (XX - e.cx) * c + (YY - e.cy) * s
        v = -(XX - e.cx) * s + (YY - e.cy) * c
        img += e.value * ((u / e.a) ** 2 + (v / e.b) ** 2 <= 1.0)
    img = img.reshape(nx, ss, ny, ss).mean(axis=(1, 3))
    return img.astype(np.complex64)


def coil_maps(rng: np.random.Generator, nx: int, ny: int, nc: int) -> np.ndarray:
    """Smooth Gaussian sensitivities normalised to ``sum_c |S_c|^2 = 1``; complex64 ``[nc][nx][ny]``."""
    X = pixel_coords(nx)[:, None]
    Y = pixel_coords(ny)[None, :]
    w = 0.4 * min(nx, ny)
    phases = rng.uniform(0.0, 2.0 * math.pi, size=nc)
    raw = np.empty((nc, nx, ny), dtype=np.complex128)
    for c in range(nc):
        px = 0.5 * nx * math.cos(2.0 * math.pi * c / nc)
        py = 0.5 * ny * math.sin(2.0 * math.pi * c / nc)
        raw[c] = np.exp(-((X - px) ** 2 + (Y - py) ** 2) / (2.0 * w * w)) * np.exp(1j * phases[c])
    norm = np.sqrt(np.sum(np.abs(raw) ** 2, axis=0))
    return (raw / norm[None]).astype(np.complex64)


def unit_noise(rng: np.random.Generator, nc: int, nk: int) -> np.ndarray:
    """Circular complex Gaussian, unit variance; complex128 ``[nc][nk]``."""
    re = rng.standard_normal((nc, nk))
    im = rng.standard_normal((nc, nk))
    return (re + 1j * im) / math.sqrt(2.0)


def add_noise(d_clean: np.ndarray, noise: np.ndarray, level: float) -> np.ndarray:
    """``d = d_clean + level * RMS(|d_clean|) * noise``, rounded to complex64."""
    d_clean = np.asarray(d_clean)
    sigma = level * math.sqrt(float(np.mean(np.abs(d_clean.astype(np.complex128)) ** 2)))
    return (d_clean.astype(np.complex128) + sigma * noise).astype(np.complex64)


@dataclasses.dataclass
class Problem:
    """One reconstruction problem.  Arrays are in the library's layouts:
    image ``[nx][ny]``, maps ``[nc][nx][ny]``, traj ``[nk][2]``, kspace ``[nc][nk]``."""
    name: str
    nx: int
    ny: int
    nc: int
    spokes: int
    readout: int
    traj: np.ndarray          # float32 [nk][2]
    image_true: np.ndarray    # complex64 [nx][ny]
    maps: np.ndarray          # complex64 [nc][nx][ny]
    noise: np.ndarray         # complex128 [nc][nk], unit variance
    noise_level: float
    lam: float
    beta: float
    admm_iters: int
    cg_iters: int
    seed: int
    rtol: float = 0.0         # Alg. 4 relative-change exit (0: fixed count)
    atol: float = 0.0         # Alg. 2 residual exit (0: fixed count)
    angles: str = "golden"    # spoke angles: "golden" or "uniform"

    @property
    def nk(self) -> int:
        return self.spokes * self.readout


def make_problem(name: str, n: int, nc: int, spokes: int, readout: int, *, seed: int,
                 golden: bool, noise_level: float, lam: float = 1e-3, beta: float = 1.0,
                 admm_iters: int = 10, cg_iters: int = 5, ny: Optional[int] = None) -> Problem:
    nx = n
    ny = n if ny is None else ny
    rng = np.random.default_rng(seed)
    ell = random_ellipses(rng, nx, ny)
    img = rasterize(ell, nx, ny)
    maps = coil_maps(rng, nx, ny, nc)
    noise = unit_noise(rng, nc, spokes * readout)
    traj = radial_trajectory(spokes, readout, golden=golden)
    return Problem(name, nx, ny, nc, spokes, readout, traj, img, maps, noise, noise_level,
                   lam, beta, admm_iters, cg_iters, seed, angles="golden" if golden else "uniform")


# The three single-reconstruction workloads (seeds fixed so that every consumer
# regenerates bit-identical inputs).
def config_small() -> Problem:
    """N=32, 4 coils, 16 uniform spokes x 64 samples, 1% noise, 10 ADMM x 5 CG."""
    return make_problem("n32_c4_s16x64", 32, 4, 16, 64, seed=1001, golden=False,
                        noise_level=0.01, lam=1e-3, beta=1.0, admm_iters=10, cg_iters=5)


def config_medium() -> Problem:
    """N=128, 12 coils, 64 golden-angle spokes x 256 samples, 0.5% noise, 30 ADMM x 8 CG."""
    return make_problem("n128_c12_s64x256", 128, 12, 64, 256, seed=1002, golden=True,
                        noise_level=0.005, lam=1e-3, beta=1.0, admm_iters=30, cg_iters=8)


def config_large() -> Problem:
    """N=256, 32 coils, 128 golden-angle spokes x 512 samples, 50 ADMM x 10 CG."""
    return make_problem("n256_c32_s128x512", 256, 32, 128, 512, seed=1003, golden=True,
                        noise_level=0.005, lam=1e-3, beta=1.0, admm_iters=50, cg_iters=10)


# The paper's own workload shapes (Section V-VI, Table I parameters, with its
# tolerance exits): a 128 x 64 grid from 13 radial readouts of 128 samples
# per coil, and a 1024 x 512 grid from 101 readouts of 1024 samples per coil
# (103,424 per coil), 12 coils each.  Uniform spoke angles: the eightfold
# undersampling keeps every eighth readout of a uniform set.
TABLE1 = dict(lam=1e-7, beta=1.0, admm_iters=5, cg_iters=20, rtol=1e-4, atol=1e-6)


def config_paper_128x64() -> Problem:
    """128 x 64 image, 12 coils, 13 x 128 samples per coil, Table I parameters."""
    p = make_problem("paper_128x64_c12_s13x128", 128, 12, 13, 128, seed=1004, golden=False, noise_level=0.005,
                     lam=TABLE1["lam"], beta=TABLE1["beta"], admm_iters=TABLE1["admm_iters"],
                     cg_iters=TABLE1["cg_iters"], ny=64)
    p.rtol, p.atol = TABLE1["rtol"], TABLE1["atol"]
    return p


def config_paper_1024x512() -> Problem:
    """1024 x 512 image, 12 coils, 101 x 1024 samples per coil, Table I parameters."""
    p = make_problem("paper_1024x512_c12_s101x1024", 1024, 12, 101, 1024, seed=1005, golden=False,
                     noise_level=0.005, lam=TABLE1["lam"], beta=TABLE1["beta"], admm_iters=TABLE1["admm_iters"],
                     cg_iters=TABLE1["cg_iters"], ny=512)
    p.rtol, p.atol = TABLE1["rtol"], TABLE1["atol"]
    return p


def batch_item(j: int) -> Problem:
    """Item ``j`` of the heterogeneous batch: N in {64,128,192,256}, coils in
    {8,16,32}, 32..200 golden-angle spokes of 2N samples, 30 ADMM x 8 CG."""
    rng = np.random.default_rng(4000 + j)
    n = int(rng.choice([64, 128, 192, 256]))
    nc = int(rng.choice([8, 16, 32]))
    spokes = int(rng.integers(32, 201))
    ell = random_ellipses(rng, n, n)
    img = rasterize(ell, n, n)
    maps = coil_maps(rng, n, n, nc)
    noise = unit_noise(rng, nc, spokes * 2 * n)
    traj = radial_trajectory(spokes, 2 * n, golden=True)
    return Problem(f"batch{j}_n{n}_c{nc}_s{spokes}", n, n, nc, spokes, 2 * n, traj, img, maps,
                   noise, 0.005, 1e-3, 1.0, 30, 8, 4000 + j)


def batch_item_shape(j: int):
    """(N, coils, spokes) of batch item ``j``: the first three draws of its
    generator, without building its phantom, maps or noise."""
    rng = np.random.default_rng(4000 + j)
    n = int(rng.choice([64, 128, 192, 256]))
    nc = int(rng.choice([8, 16, 32]))
    return n, nc, int(rng.integers(32, 201))


# A stratified subsample of the 64 batch items: two of each image size, all
# three coil counts present (item: N, coils, spokes -- 59: 64, 32, 40;
# 62: 64, 16, 57; 11: 128, 8, 77; 46: 128, 16, 120; 16: 192, 8, 52;
# 34: 192, 8, 58; 36: 256, 8, 35; 17: 256, 8, 52), within each stratum the
# items with the fewest samples (at N=128 the second is the fewest with 16
# coils, so that every coil count is present), so that the FP64 oracle
# reconstructs all eight at the full 30 x 8 steps in a few CPU-hours.
BATCH_SUBSAMPLE = (59, 62, 11, 46, 16, 34, 36, 17)


def serve_request(r: int) -> Problem:
    """Request ``r`` of the serving stream: sizes drawn as for the batch items
    (N in {64,128,192,256}, coils in {8,16,32}, 32..200 golden-angle spokes of
    2N samples, 30 ADMM x 8 CG), each with its own seeded phantom, coil maps,
    noise and trajectory (golden-angle spokes from a seeded starting angle)."""
    rng = np.random.default_rng(500000 + r)
    n = int(rng.choice([64, 128, 192, 256]))
    nc = int(rng.choice([8, 16, 32]))
    spokes = int(rng.integers(32, 201))
    rotation = float(rng.uniform(0.0, math.pi))
    ell = random_ellipses(rng, n, n)
    img = rasterize(ell, n, n)
    maps = coil_maps(rng, n, n, nc)
    noise = unit_noise(rng, nc, spokes * 2 * n)
    traj = radial_trajectory(spokes, 2 * n, golden=True, rotation=rotation)
    return Problem(f"req{r}_n{n}_c{nc}_s{spokes}", n, n, nc, spokes, 2 * n, traj, img, maps,
                   noise, 0.005, 1e-3, 1.0, 30, 8, 500000 + r)


def random_complex(rng: np.random.Generator, shape, dtype=np.complex64) -> np.ndarray:
    """Standard complex Gaussian test vector."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(dtype)
