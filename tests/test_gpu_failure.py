"""Failure detection on the device without a fault: a bounded wait that runs
out is reported as MRI_ERR_TIMEOUT through the plan's deferred status, the
status clears once read, and the context keeps working (the next operator
call gives the same result as before the timeout)."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_bounded_wait_reports_timeout(precision):
    import paper_2006_14080_gb300 as mr
    p = synth.config_small()
    traj = torch.from_numpy(p.traj).float().cuda()
    maps = torch.from_numpy(p.maps).to(torch.complex64).cuda()
    rng = np.random.default_rng(11)
    x = torch.from_numpy(synth.random_complex(rng, (p.nx, p.ny))).cuda()
    with mr.Plan(p.nx, p.ny, p.nc, traj, precision) as plan:
        before = mr.nudft_forward(plan, x, maps).cpu().numpy()
        plan.sync_status()
        plan.selftest_wait(5.0)
        with pytest.raises(mr.MriError) as ei:
            plan.sync_status()
        assert ei.value.code == mr.MRI_ERR_TIMEOUT
        plan.sync_status()  # cleared by the read
        after = mr.nudft_forward(plan, x, maps).cpu().numpy()
        plan.sync_status()
    assert np.array_equal(before, after)
    with mr.Plan(p.nx, p.ny, p.nc, traj, precision) as plan:
        for bad in (0.0, -1.0, 5000.0):
            with pytest.raises(mr.MriError) as ei:
                plan.selftest_wait(bad)
            assert ei.value.code == mr.MRI_ERR_INVALID
