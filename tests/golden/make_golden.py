"""Write the FP64 oracle's reconstructions of the seeded workloads.

Calls only ``oracle`` (and ``synth`` for the seeded inputs).  Output:
``tests/golden/admm_<name>.npz`` holding the final image ``x``, the objective
and relative-change histories, and fingerprints of the k-space input (its
L2 norm and a few samples) so that a consumer can confirm it regenerated the
same measurement.

    python tests/golden/make_golden.py small medium large3x3 batch_subsample
    python tests/golden/make_golden.py --missing batch_subsample   # only images not stored yet
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

def config_large_3x3():
    """The N=256 workload (32 coils, 128 x 512 golden-angle samples) at a reduced
    count of 3 ADMM x 3 CG steps: 12 normal operators, which the oracle finishes
    in minutes where the full 50 x 10 would take hours."""
    p = synth.config_large()
    p.admm_iters, p.cg_iters = 3, 3
    p.name = p.name + "_admm3x3"
    return p


def batch_subsample():
    """The stratified subsample of the 64-item heterogeneous batch, at the
    batch's own 30 ADMM x 8 CG steps (one file per item)."""
    return [synth.batch_item(j) for j in synth.BATCH_SUBSAMPLE]


CONFIGS = {"small": synth.config_small, "medium": synth.config_medium, "large3x3": config_large_3x3,
           "batch_subsample": batch_subsample}
SAMPLE_IDX = np.array([0, 1, 17, 1000, 4093, 16383, 123456, 196607])


def fingerprint(d):
    flat = d.reshape(-1)
    idx = SAMPLE_IDX[SAMPLE_IDX < flat.size]
    return float(np.linalg.norm(flat.astype(np.complex128))), idx, flat[idx]


def main(names, missing_only=False):
    problems = []
    for name in names:
        got = CONFIGS[name]()
        problems.extend(got if isinstance(got, list) else [got])
    for p in problems:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"admm_{p.name}.npz")
        if missing_only and os.path.exists(path):
            continue
        t0 = time.time()
        d = oracle.measurements(p)
        out = oracle.admm(p.traj, p.maps, d, p.lam, p.beta, p.admm_iters, p.cg_iters)
        norm, idx, samples = fingerprint(d)
        # images of N=256 and of the batch items are stored in complex64
        # (relative rounding 6e-8, far below the 1e-3 image bar) to keep the files small
        x = out["x"].astype(np.complex64) if (p.nx >= 256 or p.name.startswith("batch")) else out["x"]
        np.savez_compressed(path, x=x, objective=out["objective"], alpha=out["alpha"],
                            d_norm=norm, d_idx=idx, d_samples=samples,
                            lam=p.lam, beta=p.beta, admm_iters=p.admm_iters, cg_iters=p.cg_iters)
        print(f"{p.name}: {time.time() - t0:.1f} s with {oracle.get_threads()} threads -> {path}")


if __name__ == "__main__":
    args = sys.argv[1:]
    missing = "--missing" in args
    args = [a for a in args if a != "--missing"]
    main(args or ["small"], missing_only=missing)
