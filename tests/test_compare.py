"""The comparison used by the GPU parity tests (tests/compare.py), on CPU:
both its exact sort-based path and its fingerprint path (used for results
with millions of leaf points) accept any order of rows inside a leaf or a
node and reject every planted difference."""
import numpy as np
import pytest

import compare as cmp
import oracle
from paper_2302_14801_gb300 import synth


def _shuffled_within_segments(res, rng):
    """A copy of an oracle result with the rows of every leaf and of every
    node's voxel range permuted (the order both sides leave free)."""
    out = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in res.items()}
    leaf = (res["flags"] & 1) == 1
    for o, c in zip(res["point_offset"][leaf].astype(int), res["point_count"][leaf].astype(int)):
        p = rng.permutation(c) + o
        out["points"][o:o + c] = res["points"][p]
        out["index"][o:o + c] = res["index"][p]
    for o, c in zip(res["voxel_offset"].astype(int), res["voxel_count"].astype(int)):
        p = rng.permutation(c) + o
        out["voxels"][o:o + c] = res["voxels"][p]
    return out


@pytest.mark.parametrize("fast", [False, True])
def test_compare_accepts_permutations_and_rejects_mistakes(fast, monkeypatch):
    if fast:
        monkeypatch.setattr(cmp, "FAST_ROWS", 0)
    pts = synth.sphere(20_000, seed=4)
    want = oracle.build(pts, 500, 1, 21)
    rng = np.random.default_rng(1)
    got = _shuffled_within_segments(want, rng)
    cmp.compare(got, want, inp=pts)
    # a colour changed in one voxel
    bad = _shuffled_within_segments(want, rng)
    bad["voxels"][5, 1] ^= 1
    with pytest.raises(AssertionError):
        cmp.compare(bad, want, inp=pts)
    # two points swapped between two different leaves
    bad = _shuffled_within_segments(want, rng)
    leaf = np.nonzero((want["flags"] & 1) == 1)[0]
    a, b = int(want["point_offset"][leaf[0]]), int(want["point_offset"][leaf[-1]])
    bad["points"][[a, b]] = bad["points"][[b, a]]
    bad["index"][[a, b]] = bad["index"][[b, a]]
    with pytest.raises(AssertionError):
        cmp.compare(bad, want, inp=pts)
    # a voxel count moved from one cell to another of the same node
    bad = _shuffled_within_segments(want, rng)
    bad["voxels"][0, 2] += 1
    bad["voxels"][1, 2] -= 1
    with pytest.raises(AssertionError):
        cmp.compare(bad, want, inp=pts)
    # a wrong input index
    bad = _shuffled_within_segments(want, rng)
    bad["index"][3] = (bad["index"][3] + 1) % len(pts)
    with pytest.raises(AssertionError):
        cmp.compare(bad, want, inp=pts)
