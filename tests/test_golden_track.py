"""The stored oracle tracking results (tests/golden/track_oracle_*.npz) are
the oracle's: a few of their paths are tracked again here and must agree bit
for bit (no GPU needed)."""
import os
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_track_oracle as M  # noqa: E402


@pytest.mark.parametrize("name,picks", [("batched_n12_dd", (0, 1, 511, 1023)), ("stress_n10_qd", (0, 1023))])
def test_stored_oracle_tracks_reproduce(oracle_lib, name, picks):
    d = np.load(M.path(name))
    ids = d["ids"]
    assert np.array_equal(ids, M.sample_ids(name))
    sel = np.array(picks)
    o = M.track(name, ids[sel])
    assert np.array_equal(o["status"], d["status"][sel])
    assert np.array_equal(o["steps"], d["steps"][sel])
    assert np.array_equal(o["newton"], d["newton"][sel])
    assert np.array_equal(o["x_end"][:, :, 0, :], d["x_lead"][..., sel])
