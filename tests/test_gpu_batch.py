"""Batched reconstructions (one launch, heterogeneous shapes) on the GPU.

Every request of a batch must produce exactly the image it produces when
reconstructed alone: the batch only changes when kernels run, never which
kernels, tiles or summation orders compute a request.  One request is the
N=32 workload, checked against the FP64 oracle as in test_gpu_admm.
"""
import os

import numpy as np
import pytest
import torch

import fp32_floor
import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def test_batch_cache_does_not_outlive_its_plans(mr):
    """One batch reused across plans that were closed and created again, with
    the same k-space, maps and output tensors: the new plans may come back at
    the old plans' addresses, but the cached launch is keyed on each plan's
    identity and configuration, so every result equals the new plan's alone
    run, bit for bit."""
    probs = _problems()[:2]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side), mr.Batch() as batch:
        data = [(_dev(oracle.measurements(p)), _dev(p.maps)) for p in probs]
        outs = [torch.empty((p.nx, p.ny), dtype=torch.complex64, device="cuda") for p in probs]
        captures = []
        for _ in range(3):
            plans = [mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), "fp32") for p in probs]
            items = [{"plan": pl, "kspace": k, "coil_maps": m, "out": o, "lam": p.lam, "beta": p.beta,
                      "admm_iters": p.admm_iters, "cg_iters": p.cg_iters}
                     for p, pl, (k, m), o in zip(probs, plans, data, outs)]
            for o in outs:
                o.fill_(float("nan"))
            batch.reconstruct(items)
            got = [o.cpu().numpy() for o in outs]
            for it, x in zip(items, got):
                alone = mr.admm_reconstruct(it["plan"], it["kspace"], it["coil_maps"], it["lam"], it["beta"],
                                            it["admm_iters"], it["cg_iters"]).cpu().numpy()
                assert np.all(np.isfinite(x)) and np.array_equal(x, alone)
            captures.append(batch.launch_count())
            for pl in plans:
                pl.sync_status()
                pl.close()
        assert all(c > 0 for c in captures)


def _golden_item(p):
    path = os.path.join(GOLDEN, f"admm_{p.name}.npz")
    return np.load(path) if os.path.exists(path) else None


# FP32-storage floors of the subsample items, computed once for both forms
_FP32_FLOORS = {}


def _subsample_data(p):
    # the oracle's seeded measurement, as the stored oracle image was made from
    return oracle.measurements(p)


@pytest.mark.slow
def test_batch64_equals_alone_and_subsample_operators_match_oracle(mr):
    """The 64-item heterogeneous batch at its real sizes and counts (N in
    {64,128,192,256}, 8-32 coils, 32-200 spokes of 2N samples, 30 ADMM x 8 CG,
    BF16x3): every item of the batch equals its alone-run image bit for bit,
    and on the stratified subsample (two items per image size, every coil
    count) the forward and adjoint operators of each item's plan match the
    FP64 oracle at sampled outputs within the 1e-5 operator bar.  Items
    outside the subsample reconstruct seeded synthetic k-space (the oracle's
    measurement of 56 more items would take CPU-hours); the equality check
    needs no particular data."""
    sub = set(synth.BATCH_SUBSAMPLE)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        probs, items, plans, data = [], [], [], {}
        for j in range(64):
            p = synth.batch_item(j)
            d = _subsample_data(p) if j in sub else (0.05 * p.noise).astype(np.complex64)
            data[j] = d
            plan = mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), "bf16x3")
            probs.append(p)
            plans.append(plan)
            items.append({"plan": plan, "kspace": _dev(d), "coil_maps": _dev(p.maps),
                          "out": torch.full((p.nx, p.ny), float("nan"), dtype=torch.complex64, device="cuda"),
                          "lam": p.lam, "beta": p.beta, "admm_iters": p.admm_iters, "cg_iters": p.cg_iters})
        with mr.Batch() as batch:
            batch.reconstruct(items)
            batched = [it["out"].cpu().numpy() for it in items]
        alone = [mr.admm_reconstruct(it["plan"], it["kspace"], it["coil_maps"], it["lam"], it["beta"],
                                     it["admm_iters"], it["cg_iters"]).cpu().numpy() for it in items]
        ops = {}
        rng = np.random.default_rng(64)
        for j in sorted(sub):
            p, it = probs[j], items[j]
            x = synth.random_complex(rng, (p.nx, p.ny))
            ks = np.sort(rng.choice(p.nk, size=min(p.nk, 384), replace=False))
            px = np.sort(rng.choice(p.nx * p.ny, size=48, replace=False))  # flat pixel indices i*ny + j
            fwd = mr.nudft_forward(it["plan"], _dev(x), it["coil_maps"]).cpu().numpy()[:, ks]
            adj = mr.nudft_adjoint(it["plan"], it["kspace"], it["coil_maps"]).cpu().numpy().reshape(-1)[px]
            ops[j] = (x, ks, px, fwd, adj)
        for plan in plans:
            plan.sync_status()
            plan.close()
    for a, b in zip(batched, alone):
        assert np.all(np.isfinite(a)) and np.array_equal(a, b)
    for j in sorted(sub):
        p = probs[j]
        x, ks, px, fwd, adj = ops[j]
        ref_f = oracle.forward(p.traj[ks], x, p.maps)
        ref_a = oracle.adjoint_at(p.traj, data[j], p.maps, px)
        ef = np.linalg.norm(fwd - ref_f) / np.linalg.norm(ref_f)
        ea = np.linalg.norm(adj - ref_a) / np.linalg.norm(ref_a)
        print(f"{p.name}: forward {ef:.2e}, adjoint {ea:.2e} at sampled outputs")
        assert ef <= 1e-5 and ea <= 1e-5, p.name


@pytest.mark.slow
@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_batch_subsample_images_match_oracle(mr, precision):
    """The stratified subsample of the 64-item batch, reconstructed as one
    batch at the full 30 ADMM x 8 CG steps, against the FP64 oracle's images
    of the same seeded measurements (tests/golden, written by make_golden.py
    from the oracle alone): NRMSE <= 1e-3 for every item in both forms, or,
    for an item that misses it, within twice that item's FP32-storage floor
    (fp32_floor.py: the oracle's updates with exact operators and every stored
    vector rounded to complex64, the error no implementation holding its
    iterates in FP32 goes below; above 1e-3 on the 8-coil items with the
    fewest spokes per pixel)."""
    probs = [synth.batch_item(j) for j in synth.BATCH_SUBSAMPLE]
    goldens = [_golden_item(p) for p in probs]
    if any(g is None for g in goldens):
        pytest.skip("stored oracle images of the batch subsample missing (make_golden.py batch_subsample)")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        items, plans, data = [], [], []
        for p, g in zip(probs, goldens):
            d = _subsample_data(p)
            data.append(d)
            assert abs(np.linalg.norm(d.astype(np.complex128)) - float(g["d_norm"])) <= 1e-9 * float(g["d_norm"])
            plan = mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision)
            plans.append(plan)
            items.append({"plan": plan, "kspace": _dev(d), "coil_maps": _dev(p.maps),
                          "out": torch.full((p.nx, p.ny), float("nan"), dtype=torch.complex64, device="cuda"),
                          "lam": p.lam, "beta": p.beta, "admm_iters": p.admm_iters, "cg_iters": p.cg_iters})
        with mr.Batch() as batch:
            batch.reconstruct(items)
            got = [it["out"].cpu().numpy() for it in items]
        for plan in plans:
            plan.sync_status()
            plan.close()
    for p, g, x, d in zip(probs, goldens, got, data):
        ref = g["x"].astype(np.complex128)
        err = fp32_floor.nrmse(x, ref)
        bar = 1e-3
        if err > bar:
            if p.name not in _FP32_FLOORS:
                _FP32_FLOORS[p.name] = fp32_floor.nrmse(fp32_floor.reconstruct(p, d, fp32_storage=True)[0], ref)
            bar = fp32_floor.image_bar(_FP32_FLOORS[p.name])
            print(f"{p.name}: FP32-storage floor {_FP32_FLOORS[p.name]:.3e}, bar {bar:.3e}")
        print(f"{p.name} {precision}: NRMSE vs FP64 oracle = {err:.3e}")
        assert err <= bar, p.name
