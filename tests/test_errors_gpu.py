"""Failure detection without a GPU fault: bounded waits that give up, ray-front overflow,
bad inputs and calls out of order all come back as status codes."""
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


def _grid(A, n=32, value=1.0):
    t = torch.full((n, n, n), value, device="cuda", dtype=torch.float32)
    return A.Grid(t, 1.0 / n), t


def test_no_sources_is_state_error(art):
    from paper_1711_06277_gb300 import _lib as C
    g, _ = _grid(art)
    with pytest.raises(C.ArtError) as e:
        g.trace(art.Params())
    assert e.value.status == C.ART_ESTATE
    with pytest.raises(C.ArtError) as e:
        g.stats()
    assert e.value.status == C.ART_ESTATE


@pytest.mark.parametrize("kw", [dict(level0=13), dict(level0=3, level_max=2), dict(m_ray=0.0),
                                dict(tau_max=-1.0), dict(sigma_H=-1.0), dict(chunk=48),
                                dict(block_threads=100), dict(queue_capacity=2)])
def test_bad_params(art, kw):
    from paper_1711_06277_gb300 import _lib as C
    g, _ = _grid(art)
    g.add_sources([[0.5, 0.5, 0.5]], [1.0])
    with pytest.raises(C.ArtError) as e:
        g.trace(art.Params(**kw))
    assert e.value.status == C.ART_EINVAL


@pytest.mark.parametrize("pos,L", [([[0.0, 0.5, 0.5]], [1.0]), ([[0.5, 1.0, 0.5]], [1.0]),
                                   ([[0.5, 0.5, 1.5]], [1.0]), ([[0.5, 0.5, 0.5]], [-1.0]),
                                   ([[0.5, 0.5, 0.5]], [float("nan")])])
def test_bad_sources(art, pos, L):
    from paper_1711_06277_gb300 import _lib as C
    g, _ = _grid(art)
    with pytest.raises(C.ArtError) as e:
        g.add_sources(pos, L)
    assert e.value.status == C.ART_EINVAL


def test_bad_density_reported(art):
    from paper_1711_06277_gb300 import _lib as C
    g, t = _grid(art)
    t[3, 4, 5] = float("nan")
    g.add_sources([[0.5, 0.5, 0.5]], [1.0])
    with pytest.raises(C.ArtError) as e:
        g.trace(art.Params(level0=1))
    assert e.value.status == C.ART_EINVAL
    t[3, 4, 5] = -1.0
    with pytest.raises(C.ArtError):
        g.trace(art.Params(level0=1))
    t[3, 4, 5] = 1.0
    assert g.trace(art.Params(level0=1))["stats"]["status"] == 0  # usable afterwards


def test_front_overflow_reported(art):
    from paper_1711_06277_gb300 import _lib as C
    g, _ = _grid(art, n=64)
    g.add_sources([[0.5, 0.5, 0.5]], [1.0])
    with pytest.raises(C.ArtError) as e:
        g.trace(art.Params(level0=2, schedule="plain", queue_capacity=64))
    assert e.value.status == C.ART_EQUEUE_OVERFLOW
    assert g.trace(art.Params(level0=2, schedule="plain"))["stats"]["status"] == 0


def test_barrier_wait_gives_up(art):
    from paper_1711_06277_gb300 import _lib as C
    g, _ = _grid(art, n=48)
    g.add_sources(synth.uniform_positions(4, seed=1), [1.0] * 4)
    with pytest.raises(C.ArtError) as e:
        g.trace(art.Params(level0=3, wait_limit_s=-1.0))
    assert e.value.status == C.ART_ETIMEOUT
    out = g.trace(art.Params(level0=3))  # the context stays usable
    assert out["stats"]["status"] == 0 and out["stats"]["destroy"] == out["stats"]["destroy_expected"]
