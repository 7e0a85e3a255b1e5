"""The paper's own workload shapes (Section V-VI) with its Table I parameters
and tolerance exits.

128 x 64, 12 coils, 13 x 128 samples per coil: the whole reconstruction
against the FP64 oracle (same tolerance exits, same number of ADMM steps).
1024 x 512, 12 coils, 101 x 1024 samples per coil: the image is wider than
one UMMA (two 256-column parts); the operators are checked at full size on
sampled outputs (the oracle evaluates single samples and single pixels), the
reconstruction by properties (finite, non-increasing objective, the TF32 and
BF16x3 forms agree).
"""
import numpy as np
import pytest
import torch

import fp32_floor
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


def _reconstruct(mr, p, d, precision):
    with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
        obj = torch.full((p.admm_iters,), -1.0, dtype=torch.float64, device="cuda")
        alp = torch.full((p.admm_iters,), -1.0, dtype=torch.float64, device="cuda")
        x = mr.admm_reconstruct(plan, _dev(d), _dev(p.maps), p.lam, p.beta, p.admm_iters, p.cg_iters,
                                rtol=p.rtol, atol=p.atol, objective_hist=obj, alpha_hist=alp)
        plan.sync_status()
        return x.cpu().numpy(), obj.cpu().numpy(), alp.cpu().numpy()


@pytest.fixture(scope="module")
def small():
    p = synth.config_paper_128x64()
    d = oracle.measurements(p)
    ref = oracle.admm(p.traj, p.maps, d, p.lam, p.beta, p.admm_iters, p.cg_iters, rtol=p.rtol, atol=p.atol)
    return p, d, ref


@pytest.mark.parametrize("precision", ["fp32", "bf16x3", "tf32"])
def test_paper_128x64_table1_matches_oracle(mr, small, precision):
    p, d, ref = small
    x, obj, alp = _reconstruct(mr, p, d, precision)
    steps = int(np.sum(alp >= 0))
    err = _rel(x, ref["x"])
    print(f"paper 128x64 {precision}: {steps} ADMM steps (oracle {ref['steps']}), NRMSE vs FP64 oracle {err:.3e}")
    assert steps == ref["steps"]
    # This is the workload on which the paper measured its FP32-vs-FP64 ADMM
    # difference, about 1% (Section V).  With lambda = 1e-7 it is barely
    # regularised, 8x undersampled and solved 20 CG steps deep, so rounding
    # anywhere is amplified: storing the iterates in FP32 with exact operators
    # (fp32_floor.py) lands 3.7e-3 from the oracle, so the 1e-3 target is out
    # of reach for any form with FP32 vectors here.  The FP32 and BF16x3 forms
    # are held to twice that floor (fp32_floor.image_bar), inside the paper's
    # 1%.  TF32 is not FP32-equivalent (10-bit operand mantissas, ~80x the
    # FP32 form's operator error); it is held to the paper's 5%, the typical
    # error of a compressed-sensing reconstruction itself (Section V).
    if precision == "tf32":
        bar = 5e-2
    else:
        floor = fp32_floor.nrmse(fp32_floor.reconstruct(p, d, True, rtol=p.rtol, atol=p.atol)[0], ref["x"])
        bar = fp32_floor.image_bar(floor)
        print(f"paper 128x64: FP32-storage floor {floor:.3e}, bar {bar:.3e}")
    assert err <= bar


@pytest.fixture(scope="module")
def wide():
    p = synth.config_paper_1024x512()
    rng = np.random.default_rng(1024)
    kap = np.sort(rng.choice(p.nk, size=48, replace=False))
    pix = rng.choice(p.nx * p.ny, size=48, replace=False).astype(np.int32)
    y = synth.random_complex(rng, (p.nc, p.nk)).astype(np.complex128)
    x = p.image_true.astype(np.complex128)
    fwd_ref = oracle.forward(np.ascontiguousarray(p.traj[kap]), x, p.maps)  # [nc][48]
    adj_ref = oracle.adjoint_at(p.traj, y, p.maps, pix)
    return p, x, y, kap, pix, fwd_ref, adj_ref


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
def test_paper_1024x512_operators_on_sampled_outputs(mr, wide, precision):
    p, x, y, kap, pix, fwd_ref, adj_ref = wide
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
            plan.autotune(repeats=2)
            dm = _dev(p.maps)
            fwd = mr.nudft_forward(plan, _dev(x), dm).cpu().numpy()
            adj = mr.nudft_adjoint(plan, _dev(y), dm).cpu().numpy()
            plan.sync_status()
    assert _rel(fwd[:, kap], fwd_ref) <= OP_TOL[precision]
    assert _rel(adj.reshape(-1)[pix], adj_ref) <= OP_TOL[precision]


def test_paper_1024x512_reconstruction_properties(mr, wide):
    p, x, y, kap, pix, fwd_ref, adj_ref = wide
    side = torch.cuda.Stream()
    images = {}
    with torch.cuda.stream(side):
        # the measurement from the FP32 form's forward operator plus the seeded noise
        with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), "fp32") as p32:
            d = synth.add_noise(mr.nudft_forward(p32, _dev(p.image_true), _dev(p.maps)).cpu().numpy(),
                                p.noise, p.noise_level)
        for precision in ("bf16x3", "tf32"):
            img, obj, alp = _reconstruct(mr, p, d, precision)
            steps = int(np.sum(alp >= 0))
            assert 1 <= steps <= p.admm_iters
            o = obj[:steps]
            assert np.all(np.isfinite(img)) and np.all(np.isfinite(o))
            slack = 1e-3 if precision == "tf32" else 1e-5
            assert np.all(np.diff(o) <= slack * np.abs(o[:-1])), precision
            images[precision] = img
            print(f"paper 1024x512 {precision}: {steps} ADMM steps, NRMSE vs phantom {_rel(img, p.image_true):.3e}")
    assert _rel(images["tf32"], images["bf16x3"]) <= 1e-2
