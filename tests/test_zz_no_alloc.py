"""The allocation-free substep entry point (art_dt_substep_static).

It serves callers that cannot call cudaMalloc -- code inside a host framework that owns all
device memory through its own pool, or loops that cannot take cudaMalloc's implicit device
synchronization. Its scratch is a fixed array inside the library. This file is collected
last so that a failure here comes after every other test has run; it must also pass on its
own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1711_06277_gb300 import _lib as C

pytestmark = pytest.mark.gpu


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    nH = torch.from_numpy((10.0 ** rng.uniform(-1, 3, n)).astype(np.float32)).cuda()
    xn = torch.from_numpy(rng.random(n).astype(np.float32)).cuda()
    gam = torch.from_numpy((10.0 ** rng.uniform(-4, 2, n)).astype(np.float32)).cuda()
    return gam, nH, xn


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _reference(stream, n, gam, nH, xn, alpha, Cc):
    """The allocating entry point with caller scratch."""
    L = C.lib()
    scratch = torch.empty(L.art_dt_scratch_bytes(n), dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    assert L.art_dt_substep(stream, n, _p(gam), _p(nH), _p(xn), alpha, Cc, _p(scratch), _p(out)) == 0
    return out


def test_static_substep_matches_allocating_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = C.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # calls in a row with different inputs and sizes: a later call must not see an earlier
    # call's partials. The largest size fills the fixed array exactly (65,536 tiles).
    for n, seed, alpha, Cc in [(3_000_001, 1, 0.05, 0.1), (777, 2, 0.2, 0.3),
                               (C.ART_DT_STATIC_MAX_CELLS, 3, 0.1, 0.1), (1000, 4, 0.05, 0.1)]:
        gam, nH, xn = _inputs(n, seed)
        want = _reference(stream, n, gam, nH, xn, alpha, Cc)
        got = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        rc = L.art_dt_substep_static(stream, n, _p(gam), _p(nH), _p(xn), alpha, Cc, _p(got))
        assert rc == C.ART_OK
        torch.cuda.synchronize()
        assert float(got) == pytest.approx(float(want), rel=1e-5)
        assert float(got) > 0
        if n == 777:
            # and against the FP64 oracle of Eq. e:dtss, at the tolerance of the other
            # substep tests
            from oracle import oracle as O
            ref = O.dt_substep(xn.cpu().double().numpy(), gam.cpu().double().numpy(),
                               nH.cpu().double().numpy(), alpha, Cc)
            assert float(got) == pytest.approx(ref, rel=1e-5)
        del gam, nH, xn


def test_static_substep_rejects_oversize_input():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    L = C.lib()
    x = torch.zeros(4, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    n = C.ART_DT_STATIC_MAX_CELLS + 1  # checked before any work is enqueued
    rc = L.art_dt_substep_static(None, n, _p(x), _p(x), _p(x), 0.1, 0.1, _p(out))
    assert rc == C.ART_EINVAL
    assert float(out) == 0.0
