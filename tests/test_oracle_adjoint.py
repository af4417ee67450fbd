"""Pin of the oracle's reverse sweep (gradient of loss = sum_c w_c Gamma_c) by central
finite differences of the oracle's own forward trace, in FP64.

The density is stored in float32 by the library interface, so the test uses power-of-two
densities and relative steps of 2^-12, which float32 holds exactly; the log-space step is
then log(1 +- 2^-12).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def _loss(prob, w):
    r = O.trace(prob)
    return float((w * r.gamma).sum())


@pytest.mark.parametrize("dust", [False, True])
def test_adjoint_matches_finite_differences(dust):
    rng = np.random.default_rng(21)
    n = 10
    nH0 = 2.0 ** rng.integers(-3, 3, size=(n, n, n)).astype(np.float64)
    nH = 2.0 * nH0 if dust else None
    pos = rng.uniform(0.15, 0.85, size=(2, 3))
    L = np.array([0.7, 1.3])
    w = rng.random((n, n, n))
    base = dict(pos=pos, L=L, dx=1.0 / n, sigma_H=3.0, sigma_d=0.5 if dust else 0.0,
                level0=1, m_ray=4.0, tau_max=30.0, nH=nH)
    prob = O.Problem(nH0=nH0, **base)
    grad, dL, loss = O.trace_adjoint(prob, w)
    assert loss == pytest.approx(_loss(prob, w), rel=1e-12)
    d = 2.0**-12
    hp, hm = math.log1p(d), math.log1p(-d)
    gmax = np.abs(grad).max()
    cells = rng.choice(n**3, size=25, replace=False)
    for c in cells:
        k, j, i = np.unravel_index(c, (n, n, n))
        up = nH0.copy(); up[k, j, i] *= 1 + d
        dn = nH0.copy(); dn[k, j, i] *= 1 - d
        fd = (_loss(O.Problem(nH0=up, **base), w) - _loss(O.Problem(nH0=dn, **base), w)) / (hp - hm)
        assert abs(fd - grad[k, j, i]) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (c, fd, grad[k, j, i])
    for s in range(2):
        h = 1e-6
        Lp = L.copy(); Lp[s] += h
        Lm = L.copy(); Lm[s] -= h
        fd = (_loss(O.Problem(nH0=nH0, **{**base, "L": Lp}), w)
              - _loss(O.Problem(nH0=nH0, **{**base, "L": Lm}), w)) / (2 * h)
        assert dL[s] == pytest.approx(fd, rel=1e-7)


def test_adjoint_vanishes_in_vacuum_cells():
    # A cell with no neutral gas has no log n_H0 dependence at all.
    n = 8
    nH0 = np.ones((n, n, n))
    nH0[2, 3, 4] = 0.0
    prob = O.Problem(nH0=nH0, pos=[[0.5, 0.5, 0.5]], L=[1.0], dx=1.0 / n, sigma_H=2.0, level0=1)
    grad, _, _ = O.trace_adjoint(prob, np.ones((n, n, n)))
    assert grad[2, 3, 4] == 0.0
    assert np.all(grad[nH0 > 0] < 0)  # more gas in any cell shadows every later cell
