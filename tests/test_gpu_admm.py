"""End-to-end ADMM reconstructions on the GPU against the FP64 oracle.

The oracle's reconstructions of the seeded workloads are stored under
tests/golden/ by make_golden.py (which calls only the oracle).  The GPU runs
the same fixed iteration counts from the same inputs; the bar is the target
of the mixed-precision form: NRMSE <= 1e-3 of the final image against the
FP64 image, for both the plain FP32 and the BF16x3 forms.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
NRMSE_TOL = 1e-3


@pytest.fixture(scope="module")
def mr():
    import paper_2006_14080_gb300 as mr
    mr.load()
    return mr


def _dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def _golden(problem):
    path = os.path.join(GOLDEN, f"admm_{problem.name}.npz")
    if not os.path.exists(path):
        pytest.skip(f"{path} not generated")
    g = np.load(path)
    d = oracle.measurements(problem)
    # the regenerated measurement is the one the golden run used
    assert abs(np.linalg.norm(d.astype(np.complex128)) - float(g["d_norm"])) <= 1e-9 * float(g["d_norm"])
    assert np.array_equal(d.reshape(-1)[g["d_idx"]], g["d_samples"])
    return g, d


def _run(mr, p, d, precision, with_hist=True, rtol=0.0, atol=0.0, lam=None, beta=None, iters=None):
    lam = p.lam if lam is None else lam
    beta = p.beta if beta is None else beta
    admm_iters, cg_iters = (p.admm_iters, p.cg_iters) if iters is None else iters
    with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
        obj = torch.full((admm_iters,), -1.0, dtype=torch.float64, device="cuda") if with_hist else None
        alp = torch.full((admm_iters,), -1.0, dtype=torch.float64, device="cuda") if with_hist else None
        x = mr.admm_reconstruct(plan, _dev(d), _dev(p.maps), lam, beta, admm_iters, cg_iters,
                                rtol=rtol, atol=atol, objective_hist=obj, alpha_hist=alp)
        plan.sync_status()
        return (x.cpu().numpy().astype(np.complex128),
                None if obj is None else obj.cpu().numpy(), None if alp is None else alp.cpu().numpy())


def _nrmse(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


# Per-iterate bars of the N=32 workload.  The final image is held to the
# 1e-3 target for both forms.  The intermediate iterates are more sensitive
# than the final one: with 5 CG steps per x-update the second ADMM step
# amplifies the operator error of the first by about 300 in an emulation of
# the BF16x3 products (1.8e-5 NRMSE after step 1, 5.9e-3 after step 2, 5e-4
# after step 10), and by about 70 for FP32 vectors with exact operators.
# So the objective and the relative change of every step are held tightly
# for the FP32 form (emulation: 1.1e-4 and 2.3e-3 at most) and, for BF16x3,
# at the first step (operator error only) and the last.
HIST_TOL = {"fp32": {"obj": 1e-3, "alpha": 2e-2}, "bf16x3": {"obj": 1e-1, "alpha": 0.5}}


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_admm_small_matches_oracle(mr, precision):
    p = synth.config_small()
    g, d = _golden(p)
    x, obj, alp = _run(mr, p, d, precision)
    err = _nrmse(x, g["x"])
    print(f"small workload {precision}: NRMSE vs FP64 oracle = {err:.3e}")
    assert err <= NRMSE_TOL
    # histories follow the oracle's: every step within the form's bar, the
    # first (before any amplification) and the last within 1e-4 and 1e-3
    assert np.allclose(obj, g["objective"], rtol=HIST_TOL[precision]["obj"], atol=0)
    assert abs(obj[0] / g["objective"][0] - 1) <= 1e-4
    assert abs(obj[-1] / g["objective"][-1] - 1) <= NRMSE_TOL
    assert np.all(np.diff(obj) <= 1e-6 * np.abs(obj[:-1]))
    assert alp[0] == 1.0 and g["alpha"][0] == 1.0
    assert np.allclose(alp[1:], g["alpha"][1:], rtol=HIST_TOL[precision]["alpha"], atol=0)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_admm_medium_matches_oracle(mr, precision):
    p = synth.config_medium()
    g, d = _golden(p)
    x, _, _ = _run(mr, p, d, precision, with_hist=False)
    err = _nrmse(x, g["x"])
    print(f"medium workload {precision}: NRMSE vs FP64 oracle = {err:.3e}")
    assert err <= NRMSE_TOL


def test_admm_medium_tf32_reported(mr):
    # The TF32 form carries ~4e-4 relative error per operator application
    # (10-bit operand mantissas), forty times the BF16x3 form's: it fails the
    # 1e-5 operator and 1e-3 image targets, is reported as failing them, and
    # is held here only to the paper's ~1% FP32-vs-FP64 level.
    p = synth.config_medium()
    g, d = _golden(p)
    x, _, _ = _run(mr, p, d, "tf32", with_hist=False)
    err = _nrmse(x, g["x"])
    print(f"medium workload tf32: NRMSE vs FP64 oracle = {err:.3e}")
    assert err <= 1e-2


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_admm_table1_tolerances_stop_like_oracle(mr, precision):
    with open(os.path.join(GOLDEN, "table1_admm_params.json")) as fh:
        t1 = json.load(fh)
    p = synth.config_small()
    d = oracle.measurements(p)
    ref = oracle.admm(p.traj, p.maps, d, t1["lambda"], t1["beta"], t1["admm_max_iterations"],
                      t1["cg_max_iterations"], rtol=t1["admm_rtol"], atol=t1["cg_atol"])
    x, obj, alp = _run(mr, p, d, precision, lam=t1["lambda"], beta=t1["beta"],
                       iters=(t1["admm_max_iterations"], t1["cg_max_iterations"]),
                       rtol=t1["admm_rtol"], atol=t1["cg_atol"])
    steps = int(np.sum(alp >= 0))
    assert 1 <= steps <= t1["admm_max_iterations"]
    assert steps == ref["steps"]
    # Table I's lambda = 1e-7 leaves the problem barely regularised and 20 CG
    # steps deep: FP32 vector storage alone moves the FP64 solver by 1.3e-3
    # and a reordering of its FP64 sums by 4.7e-4
    # (test_table1_small_workload_amplifies_any_rounding), so the bar is the
    # paper's ~1% FP32-vs-FP64 difference (Section V)
    err = _nrmse(x, ref["x"])
    print(f"small workload, Table I parameters, {precision}: NRMSE vs FP64 oracle = {err:.3e}")
    assert err <= 1e-2


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_graph_replay_matches_direct_launches(mr, precision):
    # a side stream enables capture; the first call captures and launches the
    # graph, the second replays it, the third (graphs off) launches directly
    p = synth.config_small()
    d = oracle.measurements(p)
    side = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(side):
        with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
            dk, dm = _dev(d), _dev(p.maps)
            obj = torch.zeros(p.admm_iters, dtype=torch.float64, device="cuda")
            for graphs in (True, True, False):
                plan.set_graphs(graphs)
                x = mr.admm_reconstruct(plan, dk, dm, p.lam, p.beta, p.admm_iters, p.cg_iters,
                                        objective_hist=obj)
                outs.append((x.cpu().numpy(), obj.cpu().numpy().copy()))
            plan.sync_status()
    for x, o in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(o, outs[0][1])


def test_admm_zero_iterations_returns_zero_image(mr):
    p = synth.config_small()
    d = oracle.measurements(p)
    x, _, _ = _run(mr, p, d, "fp32", with_hist=False, iters=(0, 5))
    assert np.all(x == 0)


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_resume_continues_bit_for_bit(mr, precision):
    # (x, eta) is the whole ADMM state: 3 steps, save, 4 more from the saved
    # state = 7 steps in one call, bit for bit (direct launches and graphs)
    p = synth.config_small()
    g, d = _golden(p)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        with mr.Plan(p.nx, p.ny, p.nc, _dev(p.traj, torch.float32), precision) as plan:
            k, m = _dev(d), _dev(p.maps)
            whole, eta_whole = mr.admm_resume(plan, k, m, p.lam, p.beta, 7, p.cg_iters)
            plain = mr.admm_reconstruct(plan, k, m, p.lam, p.beta, 7, p.cg_iters)
            x3, eta3 = mr.admm_resume(plan, k, m, p.lam, p.beta, 3, p.cg_iters)
            x7, eta7 = mr.admm_resume(plan, k, m, p.lam, p.beta, 4, p.cg_iters, x0=x3.clone(), eta0=eta3.clone())
            plan.set_graphs(False)
            x7d, _ = mr.admm_resume(plan, k, m, p.lam, p.beta, 4, p.cg_iters, x0=x3.clone(), eta0=eta3.clone())
            plan.sync_status()
    assert torch.equal(whole, plain)
    assert torch.equal(x7, whole) and torch.equal(eta7, eta_whole)
    assert torch.equal(x7d, whole)
    assert not torch.equal(x3, whole)
