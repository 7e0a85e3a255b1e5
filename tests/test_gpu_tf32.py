"""The TF32 tensor-core form against an emulation of its arithmetic.

The TF32 products round every operand element to TF32 (10-bit mantissa,
nearest, ties away from zero) and accumulate in FP32.  The emulation below
forms the same real-embedded operands in numpy, rounds them the same way and
sums in FP64, so the GPU result may differ from it only by FP32 accumulation
(relative ~1e-6) and by the rare operand whose FP32 value straddles a TF32
rounding boundary differently (one term in thousands).  That separates a
correct TF32 kernel (error ~1e-6 against the emulation, ~4e-4 against the
exact operator) from a wrong one far better than the exact-operator bar.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

EMU_TOL = 2e-5


def tf32(v):
    """Round float32 values to TF32, nearest with ties away from zero."""
    b = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32)
    r = ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    return r.astype(np.float64)


def phasors(traj_axis32, n):
    # FP64 phase k * (i - n/2) reduced to [-1/2, 1/2], then the FP32 value of the phasor
    t = traj_axis32.astype(np.float64)[:, None] * (np.arange(n) - n // 2)[None, :]
    f = t - np.rint(t)
    return np.exp(-2j * np.pi * f).astype(np.complex64)


def emulate_forward(traj32, x, maps):
    ax, ay = phasors(traj32[:, 0], x.shape[0]), phasors(traj32[:, 1], x.shape[1])
    ar, ai = tf32(ax.real), tf32(ax.imag)  # [nk][nx]
    out = []
    for c in range(maps.shape[0]):
        b = (maps[c].astype(np.complex64) * x.astype(np.complex64)).astype(np.complex64)  # FP32 product
        br, bi = tf32(b.real), tf32(b.imag)  # [nx][ny]
        zr = ar @ br - ai @ bi
        zi = ai @ br + ar @ bi
        out.append(np.sum((zr + 1j * zi) * ay.astype(np.complex128), axis=1))
    return np.stack(out)


def emulate_adjoint(traj32, y, maps):
    nx, ny = maps.shape[1:]
    ax, ay = phasors(traj32[:, 0], nx), phasors(traj32[:, 1], ny)
    cr, ci = tf32(ay.real), tf32(-ay.imag)  # conj(A_y) [nk][ny]
    img = np.zeros((nx, ny), np.complex128)
    for c in range(maps.shape[0]):
        u = (np.conj(ax).T * y[c].astype(np.complex64)[None, :]).astype(np.complex64)  # [nx][nk], FP32 product
        ur, ui = tf32(u.real), tf32(u.imag)
        w = (ur @ cr - ui @ ci) + 1j * (ui @ cr + ur @ ci)
        img += np.conj(maps[c].astype(np.complex64)).astype(np.complex128) * w
    return img


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(40, 40, 3, 7, 100), (64, 48, 2, 16, 128), (100, 72, 5, 9, 61), (36, 300, 2, 4, 64)])
def test_tf32_products_match_emulation(shape):
    import paper_2006_14080_gb300 as mr
    nx, ny, nc, spokes, readout = shape
    rng = np.random.default_rng(sum(shape) + 5)
    maps = synth.coil_maps(rng, nx, ny, nc).astype(np.complex64)
    traj = synth.radial_trajectory(spokes, readout, golden=True).astype(np.float32)
    x = synth.random_complex(rng, (nx, ny))
    y = synth.random_complex(rng, (nc, traj.shape[0]))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    with mr.Plan(nx, ny, nc, dev(traj), "tf32") as plan:
        fwd = mr.nudft_forward(plan, dev(x), dev(maps)).cpu().numpy()
        adj = mr.nudft_adjoint(plan, dev(y), dev(maps)).cpu().numpy()
        plan.sync_status()
    ef, ea = emulate_forward(traj, x, maps), emulate_adjoint(traj, y, maps)
    assert _rel(fwd, ef) <= EMU_TOL
    assert _rel(adj, ea) <= EMU_TOL
    # and the emulation itself sits at TF32 distance from the exact operator
    exact_f = oracle.forward(traj.astype(np.float64), x, maps)
    assert 1e-5 < _rel(ef, exact_f) < 2e-3
