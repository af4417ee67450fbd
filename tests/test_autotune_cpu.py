"""Host logic of the launch-knob autotuner: cache keys and cache hits (no GPU needed)."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1711_06277_gb300 import art as A
from paper_1711_06277_gb300 import autotune as T


def test_cache_key_separates_workload_shapes():
    p = A.Params(level0=4, m_ray=4.0)
    keys = {T._key((64, 64, 64), 8, p), T._key((64, 64, 32), 8, p), T._key((64, 64, 64), 9, p),
            T._key((64, 64, 64), 8, A.Params(level0=3, m_ray=4.0)),
            T._key((64, 64, 64), 8, A.Params(level0=4, m_ray=2.0))}
    assert len(keys) == 5


def test_missing_or_corrupt_cache_reads_as_empty(tmp_path):
    assert T._load_cache(str(tmp_path / "none.json")) == {}
    bad = tmp_path / "bad.json"
    bad.write_text("{not json")
    assert T._load_cache(str(bad)) == {}


def test_cache_hit_returns_stored_knobs_without_timing(tmp_path):
    """A cached workload shape returns its knobs before any device work (CPU tensors here)."""
    n = 16
    nH0 = torch.ones((n, n, n))
    p = A.Params(level0=2, tau_max=30.0)
    path = tmp_path / "cache.json"
    knobs = {"chunk": 96, "block_threads": 512, "queue_capacity": 1 << 20}
    path.write_text(json.dumps({T._key(tuple(nH0.shape), 3, p): {"knobs": knobs}}))
    out = T.tune(nH0, 1.0 / n, np.full((3, 3), 0.5), np.ones(3), p, cache_path=str(path))
    assert (out.chunk, out.block_threads, out.queue_capacity) == (96, 512, 1 << 20)
    assert out.level0 == 2 and out.tau_max == 30.0
