"""The autotuner on the GPU: it times every candidate of a small space, caches the fastest
and the tuned knobs trace exactly the same rays as the library defaults."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1711_06277_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def art():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1711_06277_gb300 import art as A
    return A


def test_tune_small_space_and_cache(art, tmp_path):
    from paper_1711_06277_gb300 import autotune as T
    n = 32
    rho = torch.from_numpy(synth.lognormal_field(n, 1.5, seed=31).astype(np.float32)).cuda()
    pos = synth.uniform_positions(3, seed=31)
    L = synth.power_law_luminosities(3, seed=31)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0)
    space = {"chunk": [32, 64], "block_threads": [128, 256], "queue_capacity": [1 << 20]}
    path = str(tmp_path / "tune.json")
    tuned = T.tune(rho, 1.0 / n, pos, L, p, sample=3, space=space, cache_path=path)
    assert tuned.chunk in space["chunk"] and tuned.block_threads in space["block_threads"]
    entry = json.load(open(path))[T._key((n, n, n), 3, p)]
    assert entry["candidates"] == 4 and entry["knobs"]["chunk"] == tuned.chunk
    g = art.Grid(rho, 1.0 / n)
    g.add_sources(pos, L)
    a = g.trace(tuned, force=False)
    b = g.trace(p, force=False)
    g.close()
    assert a["stats"]["crossings"] == b["stats"]["crossings"]
    assert a["stats"]["status"] == 0 and b["stats"]["status"] == 0


def test_tune_refines_finalists_on_a_larger_sample(art, tmp_path):
    """With more sources than the first sample, the fastest candidates are timed again on
    the larger sample, and the winner is one of them."""
    from paper_1711_06277_gb300 import autotune as T
    n = 32
    rho = torch.from_numpy(synth.lognormal_field(n, 1.5, seed=32).astype(np.float32)).cuda()
    pos = synth.uniform_positions(6, seed=32)
    L = synth.power_law_luminosities(6, seed=32)
    p = art.Params(level0=3, tau_max=30.0, sigma_H=8.0)
    space = {"chunk": [32, 64, 96], "block_threads": [256], "queue_capacity": [1 << 20]}
    path = str(tmp_path / "tune.json")
    tuned = T.tune(rho, 1.0 / n, pos, L, p, sample=2, refine_sample=4, finalists=2,
                   space=space, cache_path=path)
    entry = json.load(open(path))[T._key((n, n, n), 6, p)]
    assert entry["sample_sources"] == 4 and entry["candidates"] == 3
    assert tuned.chunk in space["chunk"] and tuned.block_threads == 256
