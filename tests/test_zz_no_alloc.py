"""The allocation-free compaction entry point (ht_compact_noalloc), called
through the C ABI, gives exactly the output of ht_compact.

Some callers cannot call cudaMalloc: their memory belongs to another
framework's allocator, or a latency-critical loop must not hit the device
synchronisation cudaFree can cause.  For them the library keeps the
compaction's scratch in a fixed array instead of allocating it per call.
This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ht():
    from paper_1505_00383_gb300 import _build, ht as binding
    _build.build()
    assert torch.cuda.is_available()
    return binding


def _both(ht, status_np):
    m = status_np.size
    st = torch.from_numpy(status_np).cuda()
    out = {}
    for name, fn in (("alloc", ht.ht_compact), ("noalloc", ht.ht_compact_noalloc)):
        idx = torch.full((max(m, 1),), -7, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        fn(st, m, idx, cnt)
        c = int(cnt.item())
        out[name] = (c, idx[:c].cpu().numpy().copy())
    return out


def test_noalloc_compaction_matches_two_calls_in_a_row(ht):
    rng = synth.SplitMix64(2024)
    # two calls in a row: the second, shorter one must not see the first's indices
    for m in (70001, 1000):
        st = (rng.integers(0, 3, m) - 1).astype(np.int8)
        r = _both(ht, st)
        assert r["noalloc"][0] == r["alloc"][0] == int(np.sum(st == 0))
        assert np.array_equal(r["noalloc"][1], r["alloc"][1])


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch(ht):
    st = torch.zeros((4,), dtype=torch.int8, device="cuda")
    idx = torch.zeros((4,), dtype=torch.int32, device="cuda")
    cnt = torch.zeros((1,), dtype=torch.int32, device="cuda")
    with pytest.raises(ht.HTError) as e:
        ht.ht_compact_noalloc(st, ht.HT_NOALLOC_MAX_PATHS + 1, idx, cnt)
    assert e.value.code == ht.HT_EINVAL


def test_noalloc_empty_input_writes_only_the_count(ht):
    """m = 0: status and path_idx may be NULL; only the count (0) is written."""
    cnt = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    ht.ht_compact_noalloc(None, 0, None, cnt)
    assert int(cnt.item()) == 0


def test_noalloc_at_its_maximum_size(ht):
    """m = HT_NOALLOC_MAX_PATHS fills the scratch up to the length word; the
    result equals the allocating compaction's."""
    m = ht.HT_NOALLOC_MAX_PATHS
    st = (synth.SplitMix64(7).integers(0, 3, m) - 1).astype(np.int8)
    r = _both(ht, st)
    assert r["noalloc"][0] == r["alloc"][0] == int(np.sum(st == 0))
    assert np.array_equal(r["noalloc"][1], r["alloc"][1])
