"""The allocation-free adjoint entry point, called through the C ABI.

Some callers cannot allocate device memory (they run where the CUDA allocator
must not be touched: a real-time loop, a host callback, a process whose
device memory is reserved up front).  mri_nudft_adjoint_noalloc serves them
with a fixed, library-held scratch buffer and no plan.  Its output must match
the regular adjoint (mri_nudft_adjoint on an MRI_FP32 plan) within the FP32
operator tolerance of the other GPU tests, on two calls in a row -- the
second call reuses the scratch the first one left behind.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

FP32_OP_TOL = 2e-6


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _regular_adjoint(mr, nx, ny, nc, traj, kspace, maps):
    lib = mr.load()
    h = ctypes.c_void_p()
    assert lib.mri_plan_create(ctypes.byref(h), nx, ny, traj.shape[0], nc, ctypes.c_void_p(traj.data_ptr()),
                               mr.MRI_FP32, None) == mr.MRI_OK
    out = torch.empty((nx, ny), dtype=torch.complex64, device="cuda")
    try:
        assert lib.mri_nudft_adjoint(h, ctypes.c_void_p(kspace.data_ptr()), ctypes.c_void_p(maps.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), None) == mr.MRI_OK
        torch.cuda.synchronize()
    finally:
        lib.mri_plan_destroy(h)
    return out.cpu().numpy()


def _noalloc_adjoint(mr, nx, ny, nc, traj, kspace, maps):
    lib = mr.load()
    out = torch.full((nx, ny), float("nan"), dtype=torch.complex64, device="cuda")
    rc = lib.mri_nudft_adjoint_noalloc(nx, ny, traj.shape[0], nc, ctypes.c_void_p(traj.data_ptr()),
                                       ctypes.c_void_p(kspace.data_ptr()), ctypes.c_void_p(maps.data_ptr()),
                                       ctypes.c_void_p(out.data_ptr()), None)
    assert rc == mr.MRI_OK, lib.mri_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_adjoint_matches_regular_adjoint_twice():
    import paper_2006_14080_gb300 as mr
    cases = [(96, 80, 6, 24, 160, 21), (40, 56, 3, 7, 100, 22)]  # second call: smaller, ragged
    for nx, ny, nc, spokes, readout, seed in cases:
        rng = np.random.default_rng(seed)
        traj = _dev(synth.radial_trajectory(spokes, readout, golden=True), torch.float32)
        maps = _dev(synth.coil_maps(rng, nx, ny, nc))
        kspace = _dev(synth.random_complex(rng, (nc, traj.shape[0])))
        ref = _regular_adjoint(mr, nx, ny, nc, traj, kspace, maps)
        got = _noalloc_adjoint(mr, nx, ny, nc, traj, kspace, maps)
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) <= FP32_OP_TOL
        # and directly against the FP64 oracle's adjoint of Eq. 1
        exact = oracle.adjoint(traj.cpu().numpy(), kspace.cpu().numpy(), maps.cpu().numpy())
        assert _rel(got, exact) <= FP32_OP_TOL


def test_noalloc_adjoint_rejects_sizes_beyond_its_scratch():
    import paper_2006_14080_gb300 as mr
    lib = mr.load()
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    # 33 coils of 256 x 256 pixels need more than 16 MiB of partial images
    assert lib.mri_nudft_adjoint_noalloc(256, 256, 4, 33, p, p, p, p, None) == mr.MRI_ERR_INVALID
    assert b"scratch capacity" in lib.mri_last_error()
    # more coils than grid rows: rejected up front, not at launch
    assert lib.mri_nudft_adjoint_noalloc(1, 1, 4, 70000, p, p, p, p, None) == mr.MRI_ERR_INVALID
    assert b"65535" in lib.mri_last_error()
