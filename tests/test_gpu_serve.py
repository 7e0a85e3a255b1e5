"""Serving loop (requests from host memory under a device-memory budget).

A request's image must not depend on what else is in flight: the server runs
every request with its own plan and buffers through the same kernels as
mri_admm_reconstruct, so a request served alongside others, served alone, and
reconstructed directly through a plan give bit-identical images.  The N=32
request is also checked against the FP64 oracle (bar as in test_gpu_admm).
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
    return [
        synth.config_small(),
        synth.make_problem("s48", 48, 3, 12, 96, seed=7101, golden=True, noise_level=0.01, admm_iters=6, cg_iters=4),
        synth.make_problem("s64", 64, 6, 20, 128, seed=7102, golden=True, noise_level=0.01, admm_iters=5, cg_iters=6),
        synth.make_problem("s40", 40, 2, 9, 80, seed=7103, golden=False, noise_level=0.01, admm_iters=7,
                           cg_iters=3, ny=56),
    ]


def _submit(srv, p, d):
    return srv.submit(p.traj, d, p.maps, p.lam, p.beta, p.admm_iters, p.cg_iters)


def _direct(mr, p, d, precision):
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
            x = mr.admm_reconstruct(plan, _dev(d), _dev(p.maps), p.lam, p.beta, p.admm_iters, p.cg_iters)
            plan.sync_status()
            return x.cpu().numpy()


@pytest.mark.parametrize("precision", ["bf16x3", "fp32", "tf32"])
def test_estimate_matches_plan(mr, precision):
    for (nx, ny, nc, nk) in [(32, 32, 4, 1024), (40, 56, 2, 720), (128, 128, 12, 16384), (64, 48, 3, 999),
                             (48, 300, 2, 4096)]:
        traj = torch.zeros((nk, 2), dtype=torch.float32, device="cuda")
        with mr.Plan(nx, ny, nc, traj, precision) as plan:
            assert mr.estimate_plan_bytes(nx, ny, nk, nc, precision) == plan.device_bytes()
    assert mr.estimate_plan_bytes(0, 8, 8, 1, precision) == 0


@pytest.mark.parametrize("precision", ["bf16x3", "fp32", "tf32"])
def test_serve_mix_equals_alone(mr, precision):
    probs = _problems()
    data = [oracle.measurements(p) for p in probs]
    # every request alone (one stream, one request at a time)
    alone = []
    with mr.Server(8 << 30, max_inflight=1, precision=precision) as srv:
        for p, d in zip(probs, data):
            img, lat = srv.wait(_submit(srv, p, d))
            assert lat > 0
            alone.append(img)
    # all at once, twice over (the second round reuses cached plans), waited in reverse order
    with mr.Server(8 << 30, max_inflight=4, precision=precision) as srv:
        tickets = [_submit(srv, p, d) for _ in range(2) for p, d in zip(probs, data)]
        mixed = {t: srv.wait(t)[0] for t in reversed(tickets)}
        st = srv.stats()
        assert st["completed"] == len(tickets) and st["failed"] == 0
        assert 0 < st["p50_ms"] <= st["p99_ms"]
        assert st["peak_resident_bytes"] <= 8 << 30
    for q, t in enumerate(tickets):
        a = alone[q % len(probs)]
        assert np.all(np.isfinite(a))
        assert np.array_equal(mixed[t], a), f"request {q} differs when served alongside others"
    for q in (0, 2):
        assert np.array_equal(_direct(mr, probs[q], data[q], precision), alone[q])
    g = oracle.admm(probs[0].traj, probs[0].maps, data[0], probs[0].lam, probs[0].beta, probs[0].admm_iters,
                    probs[0].cg_iters)["x"]
    # the N=32 request against the FP64 oracle: 1e-3 for FP32 and BF16x3 as in
    # test_gpu_admm; TF32 misses that bar and is held to 5% (Section V)
    assert np.linalg.norm(alone[0] - g) / np.linalg.norm(g) <= (5e-2 if precision == "tf32" else 1e-3)


def test_serve_budget_admission(mr):
    probs = _problems()[:3]
    data = [oracle.measurements(p) for p in probs]
    need = max(mr.estimate_plan_bytes(p.nx, p.ny, p.nk, p.nc, "bf16x3") + 8 * (p.nk * p.nc + p.nc * p.nx * p.ny +
               p.nk + p.nx * p.ny) for p in probs)
    # room for one request at a time: the server must run them one after another and evict
    with mr.Server(need + 4096, max_inflight=4) as srv:
        tickets = [_submit(srv, p, d) for p, d in zip(probs, data)]
        imgs = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
        assert st["completed"] == 3 and st["peak_resident_bytes"] <= need + 4096
    with mr.Server(8 << 30, max_inflight=1) as srv:
        ref = [srv.wait(_submit(srv, p, d))[0] for p, d in zip(probs, data)]
    for a, b in zip(imgs, ref):
        assert np.array_equal(a, b)
    # a request larger than the whole budget fails on its own; the server keeps serving
    with mr.Server(1 << 20, max_inflight=2) as srv:
        big = _submit(srv, probs[2], data[2])
        with pytest.raises(mr.MriError) as ei:
            srv.wait(big)
        assert ei.value.code == mr.MRI_ERR_NOMEM
        assert srv.stats()["failed"] == 1


def test_serve_host_wait_limit(mr):
    p = synth.config_medium()
    d = oracle.measurements(p)
    with mr.Server(8 << 30, max_inflight=2) as srv:
        t = _submit(srv, p, d)
        with pytest.raises(mr.MriError) as ei:
            srv.wait(t, timeout_s=1e-4)
        assert ei.value.code == mr.MRI_ERR_TIMEOUT
        img, _ = srv.wait(t)  # the ticket is still valid
        assert np.all(np.isfinite(img))
        with pytest.raises(mr.MriError) as ei:
            srv.poll(t)  # retired
        assert ei.value.code == mr.MRI_ERR_INVALID


def test_serve_rejects_bad_requests(mr):
    with pytest.raises(mr.MriError):
        mr.Server(0)
    with mr.Server(1 << 30) as srv:
        with pytest.raises(ValueError):
            srv.submit(np.zeros((10, 2), np.float32), np.zeros((2, 9), np.complex64), np.zeros((2, 8, 8), np.complex64),
                       1e-3, 1.0, 1, 1)


def test_serve_retargets_idle_plan_of_same_shape(mr):
    # four requests of one shape with different trajectories and a budget for
    # one plan: the server must regenerate the idle plan's factors in place
    # (no allocation) and still give each request its alone result
    base = synth.make_problem("s48r", 48, 3, 12, 96, seed=7201, golden=True, noise_level=0.01,
                              admm_iters=4, cg_iters=3)
    reqs = []
    for q in range(4):
        traj = synth.radial_trajectory(12, 96, golden=True, rotation=0.37 * q)
        d = synth.add_noise(oracle.forward(traj, base.image_true, base.maps), base.noise, base.noise_level)
        reqs.append((traj, d))
    one = mr.estimate_plan_bytes(48, 48, base.nk, base.nc, "bf16x3") + \
        8 * (base.nk * base.nc + base.nc * 48 * 48 + base.nk + 48 * 48)
    with mr.Server(one + one // 2, max_inflight=2) as srv:
        tickets = [srv.submit(t, d, base.maps, base.lam, base.beta, base.admm_iters, base.cg_iters)
                   for t, d in reqs]
        tight = [srv.wait(t)[0] for t in tickets]
        assert srv.stats()["peak_resident_bytes"] <= one + one // 2
    with mr.Server(8 << 30, max_inflight=1) as srv:
        alone = [srv.wait(srv.submit(t, d, base.maps, base.lam, base.beta, base.admm_iters, base.cg_iters))[0]
                 for t, d in reqs]
    for a, b in zip(tight, alone):
        assert np.all(np.isfinite(a)) and np.array_equal(a, b)
    assert not np.array_equal(alone[0], alone[1])  # the trajectories do differ


def test_serve_keeps_maps_resident_and_replays_graphs(mr):
    # one scanner session: the same trajectory and coil maps for several
    # frames, then new maps, then a new trajectory.  One slot, so that every
    # request finds the previous one's entry idle.  The entry's factors are
    # reused from the second request on, its maps while they repeat, and its
    # reconstruction is captured as a graph at the second request and
    # replayed from the third; every image equals the direct reconstruction
    base = synth.make_problem("s48g", 48, 3, 12, 96, seed=7301, golden=True, noise_level=0.01,
                              admm_iters=4, cg_iters=3)
    rng = np.random.default_rng(7302)
    frames = [synth.add_noise(oracle.forward(base.traj, base.image_true, base.maps), synth.unit_noise(rng, base.nc,
                                                                                                      base.nk), 0.01)
              for _ in range(3)]
    maps2 = synth.coil_maps(rng, 48, 48, base.nc)
    traj2 = synth.radial_trajectory(12, 96, golden=True, rotation=0.5)
    reqs = [(base.traj, f, base.maps) for f in frames] + [(base.traj, frames[0], maps2), (traj2, frames[1], maps2)]
    with mr.Server(8 << 30, max_inflight=1) as srv:
        got = [srv.wait(srv.submit(t, d, m, base.lam, base.beta, base.admm_iters, base.cg_iters))[0]
               for t, d, m in reqs]
        st = srv.stats()
    assert st["completed"] == 5 and st["failed"] == 0
    assert st["plan_hits"] == 3          # requests 2-4 reuse the first entry's factors
    assert st["maps_reused"] == 2        # requests 2 and 3
    assert st["graph_replays"] == 2      # requests 3 and 4 (request 2 captured the graph)
    assert st["plan_retargets"] == 0     # the budget leaves room for a second entry
    for (t, d, m), img in zip(reqs, got):
        p = synth.Problem(base.name, 48, 48, base.nc, 12, 96, t, base.image_true, m, base.noise, 0.01, base.lam,
                          base.beta, base.admm_iters, base.cg_iters, base.seed)
        assert np.all(np.isfinite(img)) and np.array_equal(img, _direct(mr, p, d, "bf16x3"))
    assert not np.array_equal(got[0], got[1]) and not np.array_equal(got[0], got[3])
