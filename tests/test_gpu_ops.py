"""GPU parity of every operator of the C-ABI against the FP64 oracle.

Sizes span several tiles of both product kernels with ragged tails (image
sides not multiples of 32/64, sample counts not multiples of 64).  Bars:
relative L2 error of the DFT operators <= 2e-6 (FP32 FFMA path), <= 1e-5
(BF16x3 tensor path, the operator target) and <= 2e-3 for the TF32 tensor
path (each operand is rounded to a 10-bit mantissa, relative error up to
2^-11 = 4.9e-4 and about 2.8e-4 rms per operand, so a product term carries
about 4e-4 rms and the sum of many terms with independent errors keeps that
relative size: 2e-3 leaves a factor 5; test_gpu_tf32 checks the TF32
kernels far more tightly against an emulation of exactly that rounding).
The image-space stencils are single FP32 roundings of exact differences, so
they are held to 4 ulp of the field's maximum.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

OP_TOL = {"fp32": 2e-6, "bf16x3": 1e-5, "tf32": 2e-3}


@pytest.fixture(scope="module")
def mr():
    import paper_2006_14080_gb300 as mr
    mr.load()
    return mr


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _rel(a, b):
    a = np.asarray(a, np.complex128)
    b = np.asarray(b, np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(nx, ny, nc, spokes, readout, seed):
    rng = np.random.default_rng(seed)
    maps = synth.coil_maps(rng, nx, ny, nc)
    traj = synth.radial_trajectory(spokes, readout, golden=True)
    x = synth.random_complex(rng, (nx, ny))
    y = synth.random_complex(rng, (nc, traj.shape[0]))
    return maps, traj, x, y


SHAPES = [
    # nx, ny, nc, spokes, readout
    (40, 40, 3, 7, 100),      # ragged everywhere
    (64, 48, 2, 16, 128),     # non-square, ny a multiple of 16 only
    (100, 72, 5, 9, 61),      # odd sample count; adjoint in 128-pixel tiles (pixel-row form), rows 100-127 padding
    (200, 96, 3, 11, 90),     # two 128-pixel adjoint tiles, the second ragged
    (130, 128, 2, 8, 70),     # nx_pad 192: 64-pixel row-pair tiles at the pixel-row form's column limit
    (32, 32, 4, 16, 64),      # the small workload's shape
    (48, 300, 2, 5, 64),      # wider than one UMMA: two 256-column parts, the second mostly padding
    (40, 520, 1, 3, 50),      # three parts, one coil, ragged samples
]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_adjoint_normal_match_oracle(mr, precision, shape):
    nx, ny, nc, spokes, readout = shape
    maps, traj, x, y = _case(nx, ny, nc, spokes, readout, seed=sum(shape))
    tol = OP_TOL[precision]
    with mr.Plan(nx, ny, nc, _dev(traj, torch.float32), precision) as plan:
        dm, dx, dy = _dev(maps), _dev(x), _dev(y)
        fwd = mr.nudft_forward(plan, dx, dm).cpu().numpy()
        adj = mr.nudft_adjoint(plan, dy, dm).cpu().numpy()
        nrm = mr.normal_op(plan, dx, dm, beta=0.8).cpu().numpy()
        plan.sync_status()
    assert _rel(fwd, oracle.forward(traj, x, maps)) <= tol
    assert _rel(adj, oracle.adjoint(traj, y, maps)) <= tol
    assert _rel(nrm, oracle.normal(traj, maps, 0.8, x)) <= 2 * tol


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
def test_cartesian_grid_gives_centred_fft(mr, precision):
    n, nc = 32, 2
    rng = np.random.default_rng(3)
    maps = synth.coil_maps(rng, n, n, nc)
    x = synth.random_complex(rng, (n, n))
    traj = synth.cartesian_trajectory(n, n)
    with mr.Plan(n, n, nc, _dev(traj, torch.float32), precision) as plan:
        got = mr.nudft_forward(plan, _dev(x), _dev(maps)).cpu().numpy()
    ref = np.stack([np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(maps[c].astype(np.complex128) * x)))
                    for c in range(nc)]).reshape(nc, -1)
    assert _rel(got, ref) <= OP_TOL[precision]


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
def test_adjoint_identity_on_gpu(mr, precision):
    nx, ny, nc = 96, 80, 6
    maps, traj, x, y = _case(nx, ny, nc, 24, 160, seed=11)
    with mr.Plan(nx, ny, nc, _dev(traj, torch.float32), precision) as plan:
        dm = _dev(maps)
        fx = mr.nudft_forward(plan, _dev(x), dm).cpu().numpy().astype(np.complex128)
        fhy = mr.nudft_adjoint(plan, _dev(y), dm).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(fx, y)
    rhs = np.vdot(x, fhy)
    assert abs(lhs - rhs) <= 2 * OP_TOL[precision] * np.linalg.norm(fx) * np.linalg.norm(y)


def test_tv_pair_and_threshold_match_oracle(mr):
    rng = np.random.default_rng(5)
    for nx, ny in [(33, 47), (128, 128), (1, 5)]:
        x = synth.random_complex(rng, (nx, ny))
        g = synth.random_complex(rng, (2, nx, ny))
        gf = mr.tv_forward(_dev(x)).cpu().numpy()
        ga = mr.tv_adjoint(_dev(g)).cpu().numpy()
        ref_f = oracle.tv_forward(x)
        ref_a = oracle.tv_adjoint(g)
        assert np.abs(gf - ref_f).max() <= 4 * 2 ** -24 * 2 * np.abs(x).max()
        assert np.abs(ga - ref_a).max() <= 4 * 2 ** -24 * 4 * np.abs(g).max()
    a = synth.random_complex(rng, (5000,))
    for t in (0.0, 0.3, 1.0, 5.0):
        got = mr.soft_threshold(_dev(a), t).cpu().numpy()
        ref = oracle.shrink(a.astype(np.complex128), np.float32(t))
        assert np.abs(got - ref).max() <= 4 * 2 ** -24 * np.abs(a).max()


def test_threshold_worked_values_eq9(mr):
    import os
    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "eq9_soft_threshold.txt"), comments="#")
    for a, lam, beta, expected in rows:
        got = mr.soft_threshold(_dev(np.array([a + 0j])), lam / beta).cpu().numpy()[0]
        assert abs(got.real - expected) <= 1e-6 * max(1.0, abs(expected)) and got.imag == 0


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
def test_degenerate_shapes(mr, precision):
    # one pixel row, one coil, a single sample
    for nx, ny, nc, nk in [(1, 1, 1, 1), (3, 17, 1, 5), (70, 1, 2, 33)]:
        rng = np.random.default_rng(nx * 100 + ny)
        maps = synth.random_complex(rng, (nc, nx, ny))
        traj = rng.uniform(-0.5, 0.5, (nk, 2)).astype(np.float32)
        x = synth.random_complex(rng, (nx, ny))
        y = synth.random_complex(rng, (nc, nk))
        with mr.Plan(nx, ny, nc, _dev(traj, torch.float32), precision) as plan:
            dm = _dev(maps)
            fwd = mr.nudft_forward(plan, _dev(x), dm).cpu().numpy()
            adj = mr.nudft_adjoint(plan, _dev(y), dm).cpu().numpy()
        assert _rel(fwd, oracle.forward(traj, x, maps)) <= OP_TOL[precision]
        assert _rel(adj, oracle.adjoint(traj, y, maps)) <= OP_TOL[precision]


@pytest.mark.parametrize("shape", [(128, 128, 12), (192, 160, 6)])
def test_tile_configurations_change_schedule_not_results(mr, shape):
    # coils per forward tile and the stage counts of both operand rings change
    # the schedule only; every valid configuration must give bit-identical
    # products (same arithmetic, same order), in the pixel-row adjoint tiles
    # (128 x 128) and the row-pair ones (192 x 160)
    nx, ny, nc = shape
    maps, traj, x, y = _case(nx, ny, nc, 24, 256, seed=31)
    with mr.Plan(nx, ny, nc, _dev(traj, torch.float32), "bf16x3") as plan:
        dm, dx, dy = _dev(maps), _dev(x), _dev(y)
        ref_f = ref_a = None
        tried = set()
        for cpt in (1, 2, 3, 4):
            for fs, ast in ((f, a) for f in (2, 3, 4) for a in (2, 3, 4)):
                try:
                    plan.set_tiles(cpt, fs, ast)
                except mr.MriError:
                    continue
                tried.add((cpt, fs, ast))
                f = mr.nudft_forward(plan, dx, dm).cpu().numpy()
                a = mr.nudft_adjoint(plan, dy, dm).cpu().numpy()
                if ref_f is None:
                    ref_f, ref_a = f, a
                assert np.array_equal(f, ref_f) and np.array_equal(a, ref_a), (cpt, fs, ast)
        assert len(tried) >= 2
        if ny <= 128:  # two coils fit one 256-column tile
            assert len({t[0] for t in tried}) >= 2 and len(tried) >= 4
        with pytest.raises(mr.MriError):
            plan.set_tiles(5, 2, 2)
        cfg = plan.autotune(repeats=2)
        assert (cfg["fwd_coils_per_tile"], cfg["fwd_stages"], cfg["adj_stages"]) in tried
        assert np.array_equal(mr.nudft_forward(plan, dx, dm).cpu().numpy(), ref_f)
        plan.sync_status()
    assert _rel(ref_f, oracle.forward(traj, x, maps)) <= OP_TOL["bf16x3"]
    assert _rel(ref_a, oracle.adjoint(traj, y, maps)) <= OP_TOL["bf16x3"]


@pytest.mark.parametrize("shape", [(128, 128, 12, 64, 256), (192, 160, 6, 40, 384)])
@pytest.mark.parametrize("precision", ["bf16x3", "tf32", "fp32"])
def test_repeated_calls_and_plans_are_bit_identical(mr, precision, shape):
    # every operator sums in a fixed order, so repeating a call, or making it
    # on a second plan of the same shape, must give the same bits.  The
    # 128 x 128 image with 12 coils and 16,384 samples takes the pixel-row
    # adjoint with a dozen or more K splits per coil: the shape on which a
    # producer warp that reached its .sync.aligned TMEM stores diverged left
    # some lanes' operand rows late and changed the TF32 adjoint from call
    # to call (up to 3.6e-3 relative, rows 0-31 only).  The 192 x 160 image
    # takes the row-pair adjoint tiles instead.
    nx, ny, nc, spokes, readout = shape
    maps, traj, x, y = _case(nx, ny, nc, spokes, readout, seed=41)
    dm, dx, dy, dt = _dev(maps), _dev(x), _dev(y), _dev(traj, torch.float32)
    runs = []
    for _ in range(2):
        with mr.Plan(nx, ny, nc, dt, precision) as plan:
            a0 = mr.nudft_adjoint(plan, dy, dm).cpu().numpy()
            for _ in range(7):
                assert np.array_equal(mr.nudft_adjoint(plan, dy, dm).cpu().numpy(), a0)
            f0 = mr.nudft_forward(plan, dx, dm).cpu().numpy()
            n0 = mr.normal_op(plan, dx, dm, beta=1.0).cpu().numpy()
            assert np.array_equal(mr.normal_op(plan, dx, dm, beta=1.0).cpu().numpy(), n0)
            plan.sync_status()
        runs.append((a0, f0, n0))
    for u, v in zip(runs[0], runs[1]):
        assert np.array_equal(u, v)
    assert _rel(runs[0][0], oracle.adjoint(traj, y, maps)) <= OP_TOL[precision]


def test_invalid_arguments_are_rejected(mr):
    import ctypes
    lib = mr.load()
    h = ctypes.c_void_p()
    traj = torch.zeros((4, 2), dtype=torch.float32, device="cuda")
    assert lib.mri_plan_create(ctypes.byref(h), 0, 4, 4, 1, ctypes.c_void_p(traj.data_ptr()), 0, None) == \
        mr.MRI_ERR_INVALID
    assert lib.mri_plan_create(ctypes.byref(h), 4, 4, 4, 1, ctypes.c_void_p(traj.data_ptr()), 7, None) == \
        mr.MRI_ERR_INVALID
    assert b"precision" in lib.mri_last_error()
    with mr.Plan(8, 8, 1, traj, "fp32") as plan:
        with pytest.raises(mr.MriError) as ei:
            mr.admm_reconstruct(plan, torch.zeros((1, 4), dtype=torch.complex64, device="cuda"),
                                torch.zeros((1, 8, 8), dtype=torch.complex64, device="cuda"),
                                lam=1e-3, beta=0.0, admm_iters=1, cg_iters=1)
        assert ei.value.code == mr.MRI_ERR_INVALID


def test_tuning_table_sets_new_plans(mr, tmp_path):
    # a plan created for a shape the tuning table holds starts with its tile
    # configuration; autotune records its choice for the next plan of the same shape
    nx, ny, nc = 128, 128, 12
    maps, traj, x, y = _case(nx, ny, nc, 24, 256, seed=41)
    t = _dev(traj, torch.float32)
    nk = traj.shape[0]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    f = tmp_path / "t.json"
    f.write_text('{"format": "mrirecon-tuning", "version": 1, "entries": [{"precision": 2, "nx": %d, "ny": %d, '
                 '"nk": %d, "nc": %d, "sms": %d, "fwd_coils_per_tile": 1, "fwd_stages": 3, "adj_stages": 2}]}'
                 % (nx, ny, nk, nc, sms))
    mr.tuning_clear()
    mr.tuning_load(str(f))
    with mr.Plan(nx, ny, nc, t, "bf16x3") as plan:
        cfg = plan.config()
        assert (cfg["fwd_coils_per_tile"], cfg["fwd_stages"], cfg["adj_stages"]) == (1, 3, 2)
        tuned = plan.autotune(repeats=2)
    with mr.Plan(nx, ny, nc, t, "bf16x3") as plan:
        assert plan.config() == tuned
    mr.tuning_clear()
