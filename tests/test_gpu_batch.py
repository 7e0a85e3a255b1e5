"""Batched reconstructions (one launch, heterogeneous shapes) on the GPU.

Every request of a batch must produce exactly the image it produces when
reconstructed alone: the batch only changes when kernels run, never which
kernels, tiles or summation orders compute a request.  One request is the
N=32 workload, checked against the FP64 oracle as in test_gpu_admm.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mr():
    import paper_2006_14080_gb300 as mr
    mr.load()
    return mr


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _problems():
    small = synth.config_small()
    others = [
        synth.make_problem("b48", 48, 3, 12, 96, seed=7001, golden=True, noise_level=0.01, admm_iters=6, cg_iters=4),
        synth.make_problem("b64", 64, 6, 20, 128, seed=7002, golden=True, noise_level=0.01, admm_iters=5, cg_iters=6),
        synth.make_problem("b40", 40, 2, 9, 80, seed=7003, golden=False, noise_level=0.01, admm_iters=7,
                           cg_iters=3, ny=56),
        synth.make_problem("b96", 96, 4, 16, 192, seed=7004, golden=True, noise_level=0.005, admm_iters=4,
                           cg_iters=5),
    ]
    return [small] + others


@pytest.mark.parametrize("precision", ["bf16x3", "fp32", "tf32"])
def test_batch_equals_alone(mr, precision):
    probs = _problems()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        items, plans = [], []
        for p in probs:
            d = oracle.measurements(p)
            plan = mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision)
            plans.append(plan)
            items.append({"plan": plan, "kspace": _dev(d), "coil_maps": _dev(p.maps),
                          "out": torch.full((p.nx, p.ny), float("nan"), dtype=torch.complex64, device="cuda"),
                          "lam": p.lam, "beta": p.beta, "admm_iters": p.admm_iters, "cg_iters": p.cg_iters})
        with mr.Batch() as batch:
            batch.reconstruct(items)
            first = [it["out"].cpu().numpy() for it in items]
            batch.reconstruct(items)  # replay of the cached launch
            second = [it["out"].cpu().numpy() for it in items]
            assert batch.launch_count() > 0
        alone = []
        for it in items:
            x = mr.admm_reconstruct(it["plan"], it["kspace"], it["coil_maps"], it["lam"], it["beta"],
                                    it["admm_iters"], it["cg_iters"])
            alone.append(x.cpu().numpy())
        for plan in plans:
            plan.sync_status()
            plan.close()
    for a, b, c in zip(first, second, alone):
        assert np.all(np.isfinite(a))
        assert np.array_equal(a, b) and np.array_equal(a, c)
    # the N=32 member against the FP64 oracle: the 1e-3 image bar of
    # test_gpu_admm for FP32 and BF16x3; TF32 (10-bit operand mantissas,
    # ~4e-4 operator error) does not meet it and is held to 5%, the typical
    # error of a compressed-sensing reconstruction itself (Section V)
    g = oracle.admm(probs[0].traj, probs[0].maps, oracle.measurements(probs[0]), probs[0].lam, probs[0].beta,
                    probs[0].admm_iters, probs[0].cg_iters)["x"]
    assert np.linalg.norm(first[0] - g) / np.linalg.norm(g) <= (5e-2 if precision == "tf32" else 1e-3)


def test_batch_rejects_shared_plans(mr):
    p = synth.config_small()
    with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), "fp32") as plan, mr.Batch() as batch:
        k = torch.zeros((p.nc, p.nk), dtype=torch.complex64, device="cuda")
        m = _dev(p.maps)
        it = {"plan": plan, "kspace": k, "coil_maps": m, "lam": 1e-3, "beta": 1.0, "admm_iters": 1, "cg_iters": 1}
        with pytest.raises(mr.MriError) as ei:
            batch.reconstruct([dict(it, out=torch.empty((p.nx, p.ny), dtype=torch.complex64, device="cuda")),
                               dict(it, out=torch.empty((p.nx, p.ny), dtype=torch.complex64, device="cuda"))])
        assert ei.value.code == mr.MRI_ERR_INVALID
