"""The seeded input recipes (synth): host logic only, no GPU.

The heterogeneous batch's items are drawn from rng(4000 + j) in the order N,
coils, spokes, then phantom, maps and noise; batch_item_shape must reproduce
the first three draws without building the item, and the stratified
subsample used for parity against the oracle must cover every image size
and every coil count of the batch.
"""
import numpy as np

import synth


def test_batch_item_shape_matches_the_item():
    for j in range(64):
        n, nc, spokes = synth.batch_item_shape(j)
        rng = np.random.default_rng(4000 + j)
        assert n == int(rng.choice([64, 128, 192, 256]))
        assert nc == int(rng.choice([8, 16, 32]))
        assert spokes == int(rng.integers(32, 201))
    for j in (0, 11, 59):  # building a few items in full agrees too
        p = synth.batch_item(j)
        assert (p.nx, p.nc, p.spokes) == synth.batch_item_shape(j)
        assert p.readout == 2 * p.nx and p.traj.shape == (p.spokes * p.readout, 2)


def test_batch_subsample_is_stratified():
    sub = synth.BATCH_SUBSAMPLE
    assert len(sub) == 8 and len(set(sub)) == 8 and all(0 <= j < 64 for j in sub)
    shapes = [synth.batch_item_shape(j) for j in sub]
    assert sorted(n for n, _, _ in shapes) == [64, 64, 128, 128, 192, 192, 256, 256]
    assert {nc for _, nc, _ in shapes} == {8, 16, 32}
    # within each image size, the subsample takes the items with the fewest samples
    for n in (64, 128, 192, 256):
        stratum = sorted(((synth.batch_item_shape(j)[2], j) for j in range(64) if synth.batch_item_shape(j)[0] == n))
        picked = [j for j in sub if synth.batch_item_shape(j)[0] == n]
        assert all(synth.batch_item_shape(j)[2] <= stratum[len(stratum) // 2][0] for j in picked)
