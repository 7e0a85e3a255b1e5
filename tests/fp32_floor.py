"""The error that storing the iterates in FP32 costs by itself: an emulation
of the ADMM reconstruction (Alg. 4, with the CG of Alg. 2 as its x-update and
Eq. 8-12 as its updates) whose operators are exact to FP64 rounding and whose
stored vectors are rounded to complex64 after every update, with every
scalar (the CG step lengths, tau) kept in FP64.

Test infrastructure.  It is no part of the product and no part of the
oracle; it applies the same updates in the same order as the oracle's ADMM
(x0 = 0, eta0 = 0; mu from the shrink of Theta x + eta; b = F^H d +
(beta/2) Theta^H (mu - eta); CG warm-started at x with the residual recomputed
as b - A x; eta += Theta x' - mu), so with FP64 storage it reproduces the
oracle's image, and with complex64 storage it gives the floor that no
implementation holding x, r, p, mu, eta and A p in FP32 can go below,
however exact its operators.

The normal operator of Eq. 11 is applied through its Toeplitz structure:
(F^H F p)[n] = sum_c conj(S_c[n]) sum_m T(r_n - r_m) S_c[m] p[m], with the
point-spread kernel T(delta) = sum_kappa exp(+i 2 pi k_kappa . delta) on the
(2N_x - 1) x (2N_y - 1) lattice of pixel offsets.  The kernel is a product of
the two per-axis phasor matrices (one FP64 matrix product, phases reduced to
their fractional part as in the oracle); it is applied as a circular
convolution on the 2N_x x 2N_y grid, where the offsets of two pixels never
wrap, by FFT.  F^H d comes from the oracle.
"""
import numpy as np
from scipy import fft as _fft

import oracle


def _tv_forward(x):
    """Theta of Eq. 5: forward differences along each axis, zero past the last pixel."""
    g = np.zeros((2,) + x.shape, x.dtype)
    g[0, :-1] = x[1:] - x[:-1]
    g[0, -1] = -x[-1]
    g[1, :, :-1] = x[:, 1:] - x[:, :-1]
    g[1, :, -1] = -x[:, -1]
    return g


def _tv_adjoint(g):
    """Theta^H: the transpose of _tv_forward."""
    x = -g[0] - g[1]
    x[1:] += g[0, :-1]
    x[:, 1:] += g[1, :, :-1]
    return x


def _shrink(a, t):
    """Eq. 9 for complex entries: a (1 - t/|a|) where |a| > t, else 0."""
    m = np.abs(a)
    return np.where(m > t, a * (1.0 - t / np.maximum(m, 1e-300)), 0.0)


def _axis_phasors(k, n):
    """exp(+i 2 pi k delta) for the 2n circular offsets 0..n-1, -n..-1 of one axis."""
    delta = _fft.fftfreq(2 * n, 1.0 / (2 * n))
    t = np.outer(np.asarray(k, np.float64), delta)
    return np.exp(2j * np.pi * (t - np.rint(t)))


class NormalOperator:
    """Eq. 11, ``F^H F p + (beta/2) Theta^H Theta p``, exact to FP64 rounding."""

    def __init__(self, traj, maps, beta):
        nc, nx, ny = maps.shape
        traj = np.asarray(traj, np.float64)
        kernel = _axis_phasors(traj[:, 0], nx).T @ _axis_phasors(traj[:, 1], ny)
        kernel[nx, :] = 0.0  # offset -N never occurs between two pixels
        kernel[:, ny] = 0.0
        self.kernel_f = _fft.fft2(kernel, workers=-1)
        self.maps = np.asarray(maps, np.complex128)
        self.beta = float(beta)

    def __call__(self, p):
        nc, nx, ny = self.maps.shape
        u = np.zeros((nc, 2 * nx, 2 * ny), np.complex128)
        u[:, :nx, :ny] = self.maps * p
        v = _fft.ifft2(_fft.fft2(u, workers=-1) * self.kernel_f, workers=-1)[:, :nx, :ny]
        return np.sum(self.maps.conj() * v, axis=0) + 0.5 * self.beta * _tv_adjoint(_tv_forward(p))


class FP32Operator:
    """Eq. 11 with the DFT products in single precision: the separable
    factors A_x, A_y (Eq. 1-2, phases reduced in FP64) rounded to complex64
    and the per-coil products y_c = rowsum((A_x (S_c x)) * A_y) and
    x = sum_c conj(S_c) (A_x^H diag(y_c) conj(A_y)) taken as complex64
    matrix products with FP32 accumulation.  It stands for any FP32
    implementation of the operators, not for one kernel's summation order."""

    def __init__(self, traj, maps, beta):
        nc, nx, ny = maps.shape
        traj = np.asarray(traj, np.float64)

        def factor(k, n):
            t = np.outer(k, np.arange(n, dtype=np.float64) - n // 2)
            return np.exp(-2j * np.pi * (t - np.rint(t))).astype(np.complex64)

        self.ax = factor(traj[:, 0], nx)  # nk x nx
        ay = factor(traj[:, 1], ny)  # nk x ny
        self.ay_t = np.ascontiguousarray(ay.T)
        self.ay_conj = np.ascontiguousarray(ay.conj())
        self.ax_conj_t = np.ascontiguousarray(self.ax.conj().T)
        self.maps = np.asarray(maps, np.complex64)
        self.half_beta = np.complex64(0.5 * beta)

    def __call__(self, p):
        nc, nx, ny = self.maps.shape
        q = np.asarray(p, np.complex64)
        g = (self.maps * q).reshape(nc * nx, ny) @ self.ay_t  # (c, i) x kappa
        y = np.einsum("cik,ki->ck", g.reshape(nc, nx, -1), self.ax)
        w = (y[:, None, :] * self.ax_conj_t[None]).reshape(nc * nx, -1)
        xc = (w @ self.ay_conj).reshape(nc, nx, ny)
        out = np.sum(self.maps.conj() * xc, axis=0) + self.half_beta * _tv_adjoint(_tv_forward(q))
        return out.astype(np.complex128)


def _store64(a):
    return a


def _store32(a):
    return a.astype(np.complex64).astype(np.complex128)


def reconstruct(problem, kspace, fp32_storage, rtol=0.0, atol=0.0, fp32_operators=False):
    """Alg. 4 for ``problem`` (a synth.Problem) on the measurement ``kspace``,
    with every stored vector rounded to complex64 when ``fp32_storage``, and
    the normal operator taken in single precision (FP32Operator) when
    ``fp32_operators``.  The
    outer loop stops once the relative change ||x' - x||^2 / ||x'||^2 is at
    most rtol^2, each CG once ||r||^2 is at most atol^2, as in the oracle.
    Returns the image and the number of outer steps taken."""
    store = _store32 if fp32_storage else _store64
    op = (FP32Operator if fp32_operators else NormalOperator)(problem.traj, problem.maps, problem.beta)
    lam, beta = problem.lam, problem.beta
    fhd = store(oracle.adjoint(problem.traj, kspace, problem.maps))
    x = np.zeros(fhd.shape, np.complex128)
    eta = np.zeros((2,) + fhd.shape, np.complex128)

    def apply(p):
        return store(op(store(p)))

    steps, change = 0, 1.0
    while steps < problem.admm_iters and change > rtol * rtol:
        mu = store(_shrink(_tv_forward(x) + eta, lam / beta))
        b = store(fhd + 0.5 * beta * _tv_adjoint(mu - eta))
        xn = x.copy()
        r = store(b - apply(xn))
        d = r.copy()
        tau = np.vdot(r, r).real
        it = 0
        while it < problem.cg_iters and tau > atol * atol:
            ad = apply(d)
            alpha = tau / np.vdot(d, ad).real
            xn = store(xn + alpha * d)
            r = store(r - alpha * ad)
            tau_next = np.vdot(r, r).real
            d = store(r + (tau_next / tau) * d)
            tau = tau_next
            it += 1
        change = np.vdot(xn - x, xn - x).real / max(np.vdot(xn, xn).real, 1e-300)
        eta = store(eta + _tv_forward(xn) - mu)
        x = xn
        steps += 1
    return x, steps


def nrmse(x, ref):
    x = np.asarray(x, np.complex128)
    ref = np.asarray(ref, np.complex128)
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def image_bar(floor, target=1e-3, margin=2.0):
    """The image bar of one reconstruction: the 1e-3 target, or ``margin``
    times the FP32-storage floor where that floor is within a factor
    ``margin`` of the target or above it.  The margin covers the rounding
    pattern itself: on the N=128, 8-coil, 77-spoke batch item the floor is
    1.05e-3 with the operator applied as two per-axis matrix products and
    1.40e-3 with the Toeplitz form above, a factor 1.3 from the order of the
    FP64 operations alone."""
    return max(target, margin * floor)
