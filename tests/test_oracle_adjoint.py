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


def _loss_wv(prob, w, v):
    r = O.trace(prob)
    return float((w * r.gamma).sum() + (v * r.force).sum())


@pytest.mark.parametrize("dust", [False, True])
def test_adjoint_force_term_matches_finite_differences(dust):
    """loss = sum_c (w_c Gamma_c + v_c . f_rad,c) with v of both signs: the force part of the
    reverse sweep (q L_in e^-dtau own term, q dL in the later sums) against central
    differences of the forward trace."""
    rng = np.random.default_rng(23)
    n = 10
    nH0 = 2.0 ** rng.integers(-3, 3, size=(n, n, n)).astype(np.float64)
    nH = 2.0 * nH0 if dust else None
    pos = rng.uniform(0.15, 0.85, size=(2, 3))
    L = np.array([0.9, 0.4])
    w = 0.5 * rng.random((n, n, n))
    v = rng.uniform(-1.0, 1.0, size=(3, n, n, n))
    base = dict(pos=pos, L=L, dx=1.0 / n, sigma_H=3.0, sigma_d=0.5 if dust else 0.0,
                level0=1, m_ray=4.0, tau_max=30.0, nH=nH)
    prob = O.Problem(nH0=nH0, **base)
    grad, dL, loss = O.trace_adjoint(prob, w, v=v)
    assert loss == pytest.approx(_loss_wv(prob, w, v), rel=1e-12)
    # the force term changes the result (the pin is not vacuous)
    g0, _, _ = O.trace_adjoint(prob, w)
    assert np.abs(grad - g0).max() > 1e-3 * np.abs(grad).max()
    d = 2.0**-12
    hp, hm = math.log1p(d), math.log1p(-d)
    gmax = np.abs(grad).max()
    for c in rng.choice(n**3, size=25, replace=False):
        k, j, i = np.unravel_index(c, (n, n, n))
        up = nH0.copy(); up[k, j, i] *= 1 + d
        dn = nH0.copy(); dn[k, j, i] *= 1 - d
        fd = (_loss_wv(O.Problem(nH0=up, **base), w, v)
              - _loss_wv(O.Problem(nH0=dn, **base), w, v)) / (hp - hm)
        assert abs(fd - grad[k, j, i]) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (c, fd, grad[k, j, i])
    for s in range(2):
        h = 1e-6
        Lp = L.copy(); Lp[s] += h
        Lm = L.copy(); Lm[s] -= h
        fd = (_loss_wv(O.Problem(nH0=nH0, **{**base, "L": Lp}), w, v)
              - _loss_wv(O.Problem(nH0=nH0, **{**base, "L": Lm}), w, v)) / (2 * h)
        assert dL[s] == pytest.approx(fd, rel=1e-7)


def test_adjoint_force_term_of_a_single_axis_ray_by_hand():
    """The l0 = 0 ray along +x (exactly (1, 0, 0)) through a row of gas cells, with v = e_x
    in the row only and w = 0: beyond the source cell no other ray enters the row, so there
    f_x = dL_m / dV with closed-form dL_m, and d loss / d log n_H0[m] =
    dtau_m (L_in,m e^-dtau_m - sum_{j>m} dL_j) / dV."""
    n = 6
    px = [p for p in range(12) if np.array_equal(O.pix2vec(0, p), [1.0, 0.0, 0.0])]
    assert len(px) == 1
    row = np.array([0.5, 1.0, 2.0, 0.25, 1.5, 0.75])
    nH0 = np.zeros((n, n, n))
    nH0[2, 2, :] = row
    v = np.zeros((3, n, n, n))
    v[0, 2, 2, :] = 1.0
    dx = 1.0 / n
    prob = O.Problem(nH0=nH0, pos=[[0.5 * dx, 2.5 * dx, 2.5 * dx]], L=[1.0], dx=dx,
                     sigma_H=2.0, level0=0, level_cap=0, tau_max=1e9)
    grad, _, _ = O.trace_adjoint(prob, np.zeros((n, n, n)), v=v)
    ds = np.ones(n); ds[0] = 0.5                  # the source sits at the first cell's centre
    dtau = 2.0 * row * ds * dx
    Lin = (1.0 / 12) * np.exp(-np.concatenate([[0.0], np.cumsum(dtau)[:-1]]))
    dLs = -Lin * np.expm1(-dtau)
    dV = dx**3
    fx = O.trace(prob).force[0, 2, 2, :]
    assert np.allclose(fx[1:], dLs[1:] / dV, rtol=1e-13, atol=0)
    later = np.array([dLs[m + 1:].sum() for m in range(n)])
    expect = dtau * (Lin * np.exp(-dtau) - later) / dV
    assert np.allclose(grad[2, 2, 1:], expect[1:], rtol=1e-12, atol=0)
